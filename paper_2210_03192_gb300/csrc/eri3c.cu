// Device kernels for contracted 3-center Coulomb integrals (ab|C)
// (arXiv:2210.03192, HGPA scheme of Sec. 2.5.1):
//   pair_precompute  primitive-pair quantities gamma, P, PA, K_ab (Appendix A)
//   aux_precompute   ket primitive records
//   eri3c_kernel     per tile of (one pair, T ket shells):
//                      [00|0]^(m) from the Boys function       Sec. 2.5.2
//                      VRR1                                      Eq. vrr1
//                      CVRR2 prerequisites, contracted early     Eq. a0cv2 / Sec. 2.5.4
//                      CVRR2 targets (n-quantum form)            Sec. 2.5.4
//                      Cartesian -> solid-harmonic ket           Sec. 2.5.1
//                      HRR                                       Eq. hrr
//                      optional solid-harmonic bra, store
//
// GB300 design notes.  FP64 is the only scarce resource on this part (about
// 2 DFMA per clock per SM against 128 FFMA), so every stage is written to
// issue only the FP64 operations of the FLOP-minimal scheme with all 32 lanes
// busy, while index decoding, shared-memory traffic and table reads (integer,
// load/store pipes) hide under the FP64 pipe.  Each stage is a flat loop over
// (triple, target) items driven by host-built tables; the triple index is the
// fastest lane index when a tile holds >= 32 triples (warp-uniform table
// entries, conflict-free strided shared memory) and the target index otherwise.
// Primitive contraction happens in shared-memory accumulators (Eq. a0cv2
// prerequisites), so no intermediate CVRR2 value is ever stored to global
// memory and no atomics are needed.
#include <cuda_runtime.h>

#include "fixed128.cuh"
#include "lx3c_internal.h"

namespace lx3c {

__constant__ double c_inv2m1[32];  // 1/(2m+1)

struct FDiv {
  unsigned d, m;
  __device__ __forceinline__ void init(unsigned dd) {
    d = dd;
    m = (dd <= 1u) ? 0u : (0xFFFFFFFFu / dd + 1u);
  }
  // exact for n * d < 2^32
  __device__ __forceinline__ unsigned div(unsigned n) const { return d <= 1u ? n : __umulhi(n, m); }
};

// 1/sqrt(x) for x > 0 in FP64: single-precision seed, then one Newton-Raphson
// step carrying the second-order term (y1 = y0 (1 + e/2 + 3e^2/8),
// e = 1 - x y0^2), which takes the ~1e-7 seed error to FP64 rounding level
// with five FP64 operations.
__device__ __forceinline__ double rsqrt_fp64(double x) {
  float xf = __double2float_rn(x);
  double y0 = (double)rsqrtf(xf);
  double t = x * y0;
  double e = fma(-t, y0, 1.0);
  double p = fma(e, 0.375, 0.5);
  double q = y0 * e;
  return fma(q, p, y0);
}

// 1/x for x > 0 in FP64: single-precision seed, then two Newton-Raphson steps
// r <- r (2 - x r) written as e = 1 - x r, r <- r + r e (quadratic
// convergence: ~1e-7 -> ~1e-14 -> rounding level).
__device__ __forceinline__ double rcp_fp64(double x) {
  double r = (double)__frcp_rn(__double2float_rn(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// Compensated dot product (Ogita, Rump and Oishi's Dot2: TwoProduct by FMA,
// TwoSum, errors summed separately): about twice the working precision for
// the same result, at ~10 FP64 operations per term instead of one FMA.
// Explicitly rounded intrinsics keep the compiler from contracting the
// error-free transformations.
struct Dot2 {
  double s, c;
  __device__ __forceinline__ Dot2() : s(0.0), c(0.0) {}
  __device__ __forceinline__ void add(double a, double b) {
    const double p = __dmul_rn(a, b);
    const double ep = fma(a, b, -p);
    const double t = __dadd_rn(s, p);
    const double z = __dsub_rn(t, s);
    const double es = __dadd_rn(__dsub_rn(s, __dsub_rn(t, z)), __dsub_rn(p, z));
    s = t;
    c = __dadd_rn(c, __dadd_rn(ep, es));
  }
  __device__ __forceinline__ double value() const { return __dadd_rn(s, c); }
};

// One FP64 tensor-core step D = A B + C on an 8x8x4 tile, one warp
// (mma.sync m8n8k4 .f64).  With g = lane / 4 and q = lane % 4 the lane holds
// A[g][q], B[q][g] and the accumulator elements C[g][2q], C[g][2q+1].
__device__ __forceinline__ void dmma_8x8x4(double a, double b, double& c0, double& c1) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// pref * F_m(T) for m = hi down to lo, written to v[(m - lo) * stride].
// F_hi and exp(-T) come from the interpolation table (T < 117) or the
// asymptotic form (T >= 117, exp(-T) = 0); lower orders by the downward
// relation (2m+1) F_m = 2T F_{m+1} + exp(-T).
__device__ __forceinline__ void boys_scaled(const double* __restrict__ tab, const double* __restrict__ mid,
                                            double cL, int hi, int lo, double T, double pref, double* v,
                                            int stride) {
  double FL, ex;
  if (T < kBoysTMax) {
    int i = __float2int_rz(__double2float_rz(T) * (float)kBoysPerUnit);
    i = min(max(i, 0), kBoysNInt - 1);
    double dx = T - __ldg(mid + i);
    const double* c = tab + ((size_t)i * kBoysNF + hi) * 8;
    const double* ce = tab + ((size_t)i * kBoysNF + (kBoysNF - 1)) * 8;
    FL = __ldg(c + 7);
    ex = 0.0;
    if (hi > lo) {  // exp(-T) only feeds the downward relation
      ex = __ldg(ce + 7);
#pragma unroll
      for (int j = 6; j >= 0; --j) {
        FL = fma(FL, dx, __ldg(c + j));
        ex = fma(ex, dx, __ldg(ce + j));
      }
    } else {
#pragma unroll
      for (int j = 6; j >= 0; --j) FL = fma(FL, dx, __ldg(c + j));
    }
  } else {
    double rs = rsqrt_fp64(T);
    double b = rcp_fp64(T);
    double p = rs;
    int e = hi;
    while (e) {
      if (e & 1) p *= b;
      e >>= 1;
      if (e) b *= b;
    }
    FL = cL * p;
    ex = 0.0;
  }
  double G = pref * FL;
  v[(hi - lo) * stride] = G;
  if (hi > lo) {
    const double E = pref * ex, T2 = T + T;
    for (int m = hi - 1; m >= lo; --m) {
      G = fma(T2, G, E) * c_inv2m1[m];
      v[(m - lo) * stride] = G;
    }
  }
}

// ---------------------------------------------------------------------------
// precompute kernels
// ---------------------------------------------------------------------------


// One thread per primitive pair (pair p, a-primitive ia, b-primitive ib).
__global__ void pair_precompute(DevBasis orb, const int32_t* __restrict__ pairs, long long npair, int Ka, int Kb,
                                double* __restrict__ rec, double* __restrict__ ab, int scale_a, int scale_b) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n = npair * Ka * Kb;
  if (i >= n) return;
  long long p = i / (Ka * Kb);
  int r = (int)(i - p * Ka * Kb);
  int ia = r / Kb, ib = r - ia * Kb;
  int sa = pairs[2 * p], sb = pairs[2 * p + 1];
  const double* A = orb.xyz + 3 * sa;
  const double* B = orb.xyz + 3 * sb;
  double za = orb.exps[orb.off[sa] + ia], ca = orb.coefs[orb.off[sa] + ia];
  double zb = orb.exps[orb.off[sb] + ib], cb = orb.coefs[orb.off[sb] + ib];
  double g = za + zb, ig = 1.0 / g;
  double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
  double ab2 = AB[0] * AB[0] + AB[1] * AB[1] + AB[2] * AB[2];
  const double two_pi52 = 34.98683665524972;  // 2 pi^{5/2}
  double* o = rec + i * kPairRec;
  o[PR_G] = g;
  o[PR_K] = ca * cb * exp(-za * zb * ig * ab2) * two_pi52 * ig;
  // derivative of a primitive: d/dA phi_a = 2 za phi_{a+1} - a phi_{a-1}; the
  // 2 za factor of the first term rides on the coefficient
  if (scale_a) o[PR_K] *= 2.0 * za;
  if (scale_b) o[PR_K] *= 2.0 * zb;
  for (int x = 0; x < 3; ++x) {
    double P = (za * A[x] + zb * B[x]) * ig;
    o[PR_P + x] = P;
    o[PR_PA + x] = P - A[x];
  }
  for (int x = 0; x < 3; ++x) o[PR_PB + x] = o[PR_P + x] - B[x];
  o[PR_ZA] = za;
  o[PR_ZB] = zb;
  for (int nn = 1; nn <= 14; ++nn) o[PR_NH + nn - 1] = 0.5 * nn * ig;
  if (r == 0)
    for (int x = 0; x < 3; ++x) ab[3 * p + x] = AB[x];
}

// One thread per (ket list entry q, primitive ic): zeta_c and c_c / zeta_c.
__global__ void aux_precompute(DevBasis aux, const int32_t* __restrict__ auxs, long long naux, int Kc,
                               double* __restrict__ rec, double* __restrict__ cxyz) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= naux * Kc) return;
  long long q = i / Kc;
  int ic = (int)(i - q * Kc);
  int s = auxs[q];
  double z = aux.exps[aux.off[s] + ic], c = aux.coefs[aux.off[s] + ic];
  rec[i * kAuxRec + 0] = z;
  rec[i * kAuxRec + 1] = c / z;
  if (ic == 0)
    for (int x = 0; x < 3; ++x) cxyz[3 * q + x] = aux.xyz[3 * s + x];
}

// ---------------------------------------------------------------------------
// integral kernel
// ---------------------------------------------------------------------------

#define BUF_T(b, idx, t) ((b).base + (idx) * (b).si + (t) * (b).st)
#define BUF_TG(b, idx, g, t) ((b).base + (idx) * (b).si + (g) * (b).sg + (t) * (b).st)

// item w -> (t, x) for per-triple stages with X targets
__device__ __forceinline__ void dec2(unsigned w, int mode, const FDiv& fT, const FDiv& fX, int& t, int& x) {
  if (mode == 0) {
    unsigned q = fT.div(w);
    t = (int)(w - q * fT.d);
    x = (int)q;
  } else {
    unsigned q = fX.div(w);
    x = (int)(w - q * fX.d);
    t = (int)q;
  }
}

// item w -> (t, g, x) for per-(triple, primitive) stages
__device__ __forceinline__ void dec3(unsigned w, int mode, const FDiv& fT, const FDiv& fG, const FDiv& fX, int& t,
                                     int& g, int& x) {
  if (mode == 0) {
    unsigned q = fT.div(w);
    t = (int)(w - q * fT.d);
    unsigned r = fG.div(q);
    g = (int)(q - r * fG.d);
    x = (int)r;
  } else {
    unsigned q = fX.div(w);
    x = (int)(w - q * fX.d);
    unsigned r = fG.div(q);
    g = (int)(q - r * fG.d);
    t = (int)r;
  }
}

// Segmented dot products out[o] += sum_{r < len} prod(o, r) for o < nout,
// each partial result handed to emit(o, value), which adds it to global
// memory with an atomic (whole: one lane per output, each emitted once).  The FP64 pipe charges a whole warp instruction
// whatever the number of active lanes, and one lane's dependent FMAs are
// serialised, so the mapping follows the estimated chain length: one lane per
// output (two partial sums) when there are many outputs, else one warp per
// (output, 128-term chunk) whose lanes each emit their own partial sum (a warp
// shuffle reduction here costs the whole kernel registers).
template <class Prod, class Emit>
__device__ __forceinline__ void seg_dot(int nout, int len, const Prod& prod, const Emit& emit, bool whole = false) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kThreads / 32, kChunk = 128;
  if (nout <= 0 || len <= 0) return;
  const int nch = (len + kChunk - 1) / kChunk;
  const long long lane_steps = (long long)((nout + kThreads - 1) / kThreads) * ((len + 1) / 2);
  const long long warp_steps = (long long)((nout * nch + kWarps - 1) / kWarps) * ((min(len, kChunk) + 31) / 32 + 1);
  if (whole || lane_steps <= warp_steps) {
    for (int o = tid; o < nout; o += kThreads) {
      double s0 = 0.0, s1 = 0.0;
      int r = 0;
      for (; r + 1 < len; r += 2) {
        s0 = prod(o, r, s0);
        s1 = prod(o, r + 1, s1);
      }
      if (r < len) s0 = prod(o, r, s0);
      emit(o, s0 + s1);
    }
  } else {
    for (int it = warp; it < nout * nch; it += kWarps) {
      const int o = it / nch, r0 = (it - o * nch) * kChunk, r1 = min(len, r0 + kChunk);
      if (r0 + lane >= r1) continue;
      double s = 0.0;
      for (int r = r0 + lane; r < r1; r += 32) s = prod(o, r, s);
      emit(o, s);
    }
  }
}

// HRR rounds (Eq. hrr; Sec. 2.5.5 for two-quantum rounds) and the optional
// solid-harmonic bra transforms on tv triples of H[0]; returns the buffer
// holding the final block.
__device__ __forceinline__ Buf hrr_and_bra(const ClassDesc& d, double* sm, int T, int tv, int mode, const FDiv& fT) {
  const unsigned tid = threadIdx.x;
  // ---- HRR (Eq. hrr) round by round: each row is dst = sum_t coef_t src_t
  // over 2 terms (one quantum moved, Eq. hrr) or 3-4 terms (two quanta,
  // Sec. 2.5.5), the coefficients products of AB components
  for (int j = 1; j <= d.nhrr; ++j) {
    FDiv fX, fC;
    const int nx = d.hrows[j] * d.nC;
    fX.init(nx);
    fC.init(d.nC);
    const unsigned n = (unsigned)(T * nx);
    const Buf hi = d.H[j - 1], ho = d.H[j];
    const double* abp = sm + d.ab_base;
    for (unsigned w = tid; w < n; w += kThreads) {
      int t, x;
      dec2(w, mode, fT, fX, t, x);
      if (t >= tv) continue;
      const int r = (int)fC.div(x), C = x - r * d.nC;
      const uint4 e = __ldg(d.htab + d.hstart[j] + r);
      const unsigned nt = e.x >> 16;
      double v = fma(abp[(e.w >> 4) & 0xF], sm[BUF_T(hi, (int)(e.y >> 16) * d.nC + C, t)],
                     sm[BUF_T(hi, (int)(e.y & 0xFFFF) * d.nC + C, t)]);
      if (nt > 2) v = fma(abp[(e.w >> 8) & 0xF], sm[BUF_T(hi, (int)(e.z & 0xFFFF) * d.nC + C, t)], v);
      if (nt > 3) v = fma(abp[(e.w >> 12) & 0xF], sm[BUF_T(hi, (int)(e.z >> 16) * d.nC + C, t)], v);
      sm[BUF_T(ho, (int)(e.x & 0xFFFF) * d.nC + C, t)] = v;
    }
    __syncthreads();
  }
  // ---- optional solid-harmonic bra
  Buf cur = d.H[d.nhrr];
  if (d.nbA) {
    FDiv fX, fC, fB;
    const int nx = d.nbA * d.nC;
    fX.init(nx);
    fC.init(d.nC);
    fB.init(d.ncB);
    const unsigned n = (unsigned)(T * nx);
    for (unsigned w = tid; w < n; w += kThreads) {
      int t, x;
      dec2(w, mode, fT, fX, t, x);
      if (t >= tv) continue;
      const int row = (int)fC.div(x), C = x - row * d.nC;
      const int A = (int)fB.div(row), ib = row - A * d.ncB;
      const int q0 = __ldg(d.baptr + A), q1 = __ldg(d.baptr + A + 1);
      double s;
      const int2 e0 = __ldg(d.baent + q0);
      if (q1 - q0 == 1 && e0.y == 0) {
        s = sm[BUF_T(cur, (e0.x * d.ncB + ib) * d.nC + C, t)];
      } else {
        s = 0.0;
        for (int q = q0; q < q1; ++q) {
          const int2 e = __ldg(d.baent + q);
          s = fma(__ldg(d.pal + e.y), sm[BUF_T(cur, (e.x * d.ncB + ib) * d.nC + C, t)], s);
        }
      }
      sm[BUF_T(d.BA, x, t)] = s;
    }
    __syncthreads();
    cur = d.BA;
  }
  if (d.nbB) {
    // items B-slowest in mode 1: a warp's lanes share B's trip count
    FDiv fX, fC, fB, fAC;
    const int nx = d.nbB * d.nC;
    const int nBs = d.nB, nAC = (d.nbB / d.nB) * d.nC;
    fX.init(nx);
    fC.init(d.nC);
    fB.init(nBs);
    fAC.init(nAC);
    const unsigned n = (unsigned)(T * nx);
    for (unsigned w = tid; w < n; w += kThreads) {
      int t, x;
      dec2(w, mode, fT, fX, t, x);
      if (t >= tv) continue;
      int A, B, C;
      if (mode == 0) {
        const int row = (int)fC.div(x);
        C = x - row * d.nC;
        A = (int)fB.div(row);
        B = row - A * nBs;
      } else {
        B = (int)fAC.div(x);
        const int rem = x - B * nAC;
        A = (int)fC.div(rem);
        C = rem - A * d.nC;
      }
      x = (A * nBs + B) * d.nC + C;
      const int q0 = __ldg(d.bbptr + B), q1 = __ldg(d.bbptr + B + 1);
      double s;
      const int2 e0 = __ldg(d.bbent + q0);
      if (q1 - q0 == 1 && e0.y == 0) {
        s = sm[BUF_T(cur, (A * d.ncB + e0.x) * d.nC + C, t)];
      } else {
        s = 0.0;
        for (int q = q0; q < q1; ++q) {
          const int2 e = __ldg(d.bbent + q);
          s = fma(__ldg(d.pal + e.y), sm[BUF_T(cur, (A * d.ncB + e.x) * d.nC + C, t)], s);
        }
      }
      sm[BUF_T(d.BB, x, t)] = s;
    }
    __syncthreads();
    cur = d.BB;
  }
  return cur;
}

// One tile: (sub-pair, up to T ket shells) through every stage, ending in the
// store, the DF-J digestion or the gradient digestion.  kVar selects the
// instantiation: 0 the plain kernel (store, per-integral DF-J and gradient
// digestion), 1 adds the several-density digestion on FP64 tensor-core
// tiles (digest == 4), 2 the contraction at the (e 0|c) level (digest ==
// 5), each in a kernel of its own so that the plain launches keep their
// register count.
template <int kVar>
__device__ __forceinline__ void tile_body(const ClassDesc& d, long long tile, double* sm) {
  const unsigned tid = threadIdx.x;
  const int T = d.T, G = d.G, mode = d.mode, lc = d.lc, Lab = d.Lab;
  FDiv fT, fG, fKc;
  fT.init(T);
  fG.init(G);
  fKc.init(d.Kc);
  const int auxsz = 3 + kAuxRec * d.Kc;
  {
    long long sub;
    int aux0, tv;
    if (d.tiles) {
      const int4 tt = __ldg(d.tiles + tile);
      sub = tt.x;
      aux0 = tt.y;
      tv = tt.z;
    } else {
      sub = tile / d.ntile_aux;
      aux0 = (int)(tile - sub * d.ntile_aux) * T;
      tv = (int)min((long long)T, d.naux - aux0);
    }
    const int4 sp = __ldg(d.subpairs + sub);
    const long long pair = sp.x;
    const int kab = sp.z, accum = sp.w;
    if (kab == 0) return;  // a sub-pair without primitive pairs adds nothing (uniform across the CTA)
    const int K = kab * d.Kc;
    const int nchunk = (K + G - 1) / G;
    __syncthreads();  // previous tile done with shared memory
    {
      // this sub-pair's primitive-pair records, in its orientation
      for (int i = tid; i < kab * kPairRec; i += kThreads) {
        const int g = i / kPairRec, f = i - g * kPairRec;
        int fs = f;
        if (d.orient) {
          if (f >= PR_PA && f < PR_PA + 3) fs = f + (PR_PB - PR_PA);
          else if (f == PR_ZA) fs = PR_ZB;
          else if (f == PR_ZB) fs = PR_ZA;
        }
        const long long r = pair * d.Kab_rec + __ldg(d.primidx + sp.y + g);
        sm[d.pair_base + i] = d.pairrec[r * kPairRec + fs];
      }
      if (tid < 13) {
        // the HRR coefficients: 1, AB_i, 2 AB_i, AB_i^2, AB_x AB_y, AB_x AB_z, AB_y AB_z
        const double sg = d.orient ? -1.0 : 1.0;
        const double x = sg * d.pairab[pair * 3], y = sg * d.pairab[pair * 3 + 1], z = sg * d.pairab[pair * 3 + 2];
        const int ax = tid >= 1 && tid <= 9 ? (int)(tid - 1) % 3 : 0;
        const double u = ax == 0 ? x : (ax == 1 ? y : z);
        double v = 1.0;
        if (tid >= 1 && tid <= 3) v = u;
        else if (tid >= 4 && tid <= 6) v = 2.0 * u;
        else if (tid >= 7 && tid <= 9) v = u * u;
        else if (tid == 10) v = x * y;
        else if (tid == 11) v = x * z;
        else if (tid == 12) v = y * z;
        sm[d.ab_base + tid] = v;
      }
      for (int i = tid; i < tv * auxsz; i += kThreads) {
        int t = i / auxsz, r = i - t * auxsz;
        sm[d.aux_base + i] = r < 3 ? d.auxc[(long long)(aux0 + t) * 3 + r]
                                   : d.auxrec[(long long)(aux0 + t) * d.Kc * kAuxRec + (r - 3)];
      }
      FDiv fA;
      fA.init(d.NACC);
      for (unsigned w = tid; w < (unsigned)(T * d.NACC); w += kThreads) {
        int t, a;
        dec2(w, mode, fT, fA, t, a);
        sm[BUF_T(d.P, a, t)] = 0.0;
      }
    }
    __syncthreads();

    for (int chunk = 0; chunk < nchunk; ++chunk) {
      const int p0 = chunk * G;
      const int gcnt = min(G, K - p0);
      // ---- stage A: geometry, Boys function, [00|0]^(m) and recurrence factors
      for (unsigned w = tid; w < (unsigned)(T * G); w += kThreads) {
        int t, g;
        if (mode == 0) {
          unsigned q = fT.div(w);
          t = (int)(w - q * T);
          g = (int)q;
        } else {
          unsigned q = fG.div(w);
          g = (int)(w - q * G);
          t = (int)q;
        }
        if (t >= tv || g >= gcnt) continue;
        const int p = p0 + g;
        const int ip = (int)fKc.div(p), ic = p - ip * d.Kc;
        const double* pr = sm + d.pair_base + ip * kPairRec;
        const double* ax = sm + d.aux_base + t * auxsz;
        const double gam = pr[PR_G], zc = ax[3 + kAuxRec * ic], ccp = ax[4 + kAuxRec * ic];
        const double s = gam + zc;
        const double rs = rsqrt_fp64(s);
        const double r = rs * rs;
        const double rg = zc * r;    // rho / gamma
        const double gr = gam * r;   // rho / zeta_c
        const double PCx = pr[PR_P] - ax[0], PCy = pr[PR_P + 1] - ax[1], PCz = pr[PR_P + 2] - ax[2];
        const double pc2 = fma(PCz, PCz, fma(PCy, PCy, PCx * PCx));
        const double rho = gam * rg;
        const double Tb = rho * pc2;
        const double pref = pr[PR_K] * ccp * rs;
        const int fb = BUF_TG(d.F, 0, g, t);
        const int fs = d.F.si;
        if (Lab > 0) {  // VRR1 factors (rho/gamma) PC
          sm[fb] = rg * PCx;
          sm[fb + fs] = rg * PCy;
          sm[fb + 2 * fs] = rg * PCz;
        }
        sm[fb + 3 * fs] = rg;
        if (lc > 0) {
          double X[3] = {gr * PCx, gr * PCy, gr * PCz};
          for (int i = 0; i < 3; ++i) {
            double v = X[i];
            sm[fb + (4 + i * lc) * fs] = v;
            for (int j = 2; j <= lc; ++j) {
              v *= X[i];
              sm[fb + (4 + i * lc + j - 1) * fs] = v;
            }
          }
          double Y = 0.5 * r, v = Y;
          sm[fb + (4 + 3 * lc) * fs] = v;
          for (int k = 2; k <= lc; ++k) {
            v *= Y;
            sm[fb + (4 + 3 * lc + k - 1) * fs] = v;
          }
        }
        boys_scaled(d.boys_tab, d.boys_mid, d.boys_cL, d.L, lc, Tb, pref, sm + BUF_TG(d.V, 0, g, t), d.V.si);
      }
      __syncthreads();
      // ---- weights W_{k,n} = Y^k X^n (Eq. a0cv2)
      {
        FDiv fX;
        fX.init(d.nW);
        const unsigned n = (unsigned)(T * G * d.nW);
        for (unsigned w = tid; w < n; w += kThreads) {
          int t, g, x;
          dec3(w, mode, fT, fG, fX, t, g, x);
          if (t >= tv || g >= gcnt) continue;
          const int4 it = __ldg(d.wtab + x);
          const int dst = it.x & 0xFFFF, cnt = it.z >> 16;
          const int fb = BUF_TG(d.F, 0, g, t), fs = d.F.si;
          double v = 1.0;
          if (cnt > 0) v = sm[fb + (it.x >> 16) * fs];
          if (cnt > 1) v *= sm[fb + (it.y & 0xFFFF) * fs];
          if (cnt > 2) v *= sm[fb + (it.y >> 16) * fs];
          if (cnt > 3) v *= sm[fb + (it.z & 0xFFFF) * fs];
          sm[BUF_TG(d.W, dst, g, t)] = v;
        }
      }
      // ---- VRR1, level by level (Eq. vrr1)
      for (int e = 1; e <= Lab; ++e) {
        const int j0 = d.vlev_start[e - 1];
        const int nl = d.vlev_start[e] - j0;
        FDiv fX;
        fX.init(nl);
        const unsigned n = (unsigned)(T * G * nl);
        for (unsigned w = tid; w < n; w += kThreads) {
          int t, g, x;
          dec3(w, mode, fT, fG, fX, t, g, x);
          if (t >= tv || g >= gcnt) continue;
          const uint4 it = __ldg(d.vtab + j0 + x);
          const int dst = it.x & 0xFFFF, a = it.x >> 16, an = it.y & 0xFFFF, b = it.y >> 16, bn = it.z & 0xFFFF;
          const int axis = (it.z >> 16) & 0xF, nq = (it.z >> 20) & 0xF;
          const int p = p0 + g;
          const int ip = (int)fKc.div(p);
          const double* pr = sm + d.pair_base + ip * kPairRec;
          const int vb = BUF_TG(d.V, 0, g, t), vs = d.V.si;
          const int fb = BUF_TG(d.F, 0, g, t), fs = d.F.si;
          double val = pr[PR_PA + axis] * sm[vb + a * vs];
          val = fma(-sm[fb + axis * fs], sm[vb + an * vs], val);
          if (nq) {
            double u = fma(-sm[fb + 3 * fs], sm[vb + bn * vs], sm[vb + b * vs]);
            val = fma(pr[PR_NH + nq - 1], u, val);
          }
          sm[vb + dst * vs] = val;
        }
        __syncthreads();
      }
      if (Lab == 0) __syncthreads();
      // ---- accumulate CVRR2 prerequisites over the chunk's primitives; two
      // independent accumulators per thread keep two FMA chains in flight
      {
        FDiv fX;
        fX.init(d.NACC);
        const unsigned n = (unsigned)(T * d.NACC);
        for (unsigned w0 = tid; w0 < n; w0 += 2 * kThreads) {
          const unsigned w1 = w0 + kThreads;
          const bool has1 = w1 < n;
          int t0, a0, t1, a1;
          dec2(w0, mode, fT, fX, t0, a0);
          dec2(has1 ? w1 : w0, mode, fT, fX, t1, a1);
          const bool ok0 = t0 < tv, ok1 = has1 && t1 < tv;
          const unsigned e0 = __ldg(d.atab + a0), e1 = __ldg(d.atab + a1);
          const int pa0 = BUF_T(d.P, a0, t0), pa1 = BUF_T(d.P, a1, t1);
          const int vb0 = BUF_TG(d.V, (int)(e0 & 0xFFFF), 0, t0), wb0 = BUF_TG(d.W, (int)(e0 >> 16), 0, t0);
          const int vb1 = BUF_TG(d.V, (int)(e1 & 0xFFFF), 0, t1), wb1 = BUF_TG(d.W, (int)(e1 >> 16), 0, t1);
          // FP64 instructions cost a whole warp slot, so only stored chains run
          if (ok0 && ok1) {
            double acc0 = sm[pa0], acc1 = sm[pa1];
#pragma unroll 4
            for (int g = 0; g < gcnt; ++g) {
              acc0 = fma(sm[vb0 + g * d.V.sg], sm[wb0 + g * d.W.sg], acc0);
              acc1 = fma(sm[vb1 + g * d.V.sg], sm[wb1 + g * d.W.sg], acc1);
            }
            sm[pa0] = acc0;
            sm[pa1] = acc1;
          } else if (ok0 || ok1) {
            const int pa = ok0 ? pa0 : pa1, vb = ok0 ? vb0 : vb1, wb = ok0 ? wb0 : wb1;
            double acc = sm[pa];
#pragma unroll 4
            for (int g = 0; g < gcnt; ++g) acc = fma(sm[vb + g * d.V.sg], sm[wb + g * d.W.sg], acc);
            sm[pa] = acc;
          }
        }
      }
      __syncthreads();
    }

    // ---- CVRR2 targets (a 0|c) by the n-quantum gather (Sec. 2.5.4)
    {
      FDiv fX;
      fX.init(d.ngt);
      const unsigned n = (unsigned)(T * d.ngt);
      for (unsigned w = tid; w < n; w += kThreads) {
        int t, r;
        dec2(w, mode, fT, fX, t, r);
        if (t >= tv) continue;
        const int id = __ldg(d.gdst + r);
        double s = 0.0;
        if (d.comp & 1) {
          const int q0 = __ldg(d.gptr + id), q1 = __ldg(d.gptr + id + 1);
          Dot2 acc;
          for (int q = q0; q < q1; ++q) {
            const unsigned e = __ldg(d.gterm + q);
            acc.add(__ldg(d.pal + (e >> 20)), sm[BUF_T(d.P, e & 0xFFFFF, t)]);
          }
          s = acc.value();
        } else if (mode == 0) {
          // lanes share the target: CSR row, broadcast loads
          const int q0 = __ldg(d.gptr + id), q1 = __ldg(d.gptr + id + 1);
#pragma unroll 4
          for (int q = q0; q < q1; ++q) {
            const unsigned e = __ldg(d.gterm + q);
            s = fma(__ldg(d.pal + (e >> 20)), sm[BUF_T(d.P, e & 0xFFFFF, t)], s);
          }
        } else {
          // lanes take consecutive targets: sliced ELL, one coalesced line
          // per term step and one trip count per slice
          const int2 sl = __ldg(d.gslice + (r >> 5));
          const unsigned* ge = d.gell + sl.x + (r & 31);
#pragma unroll 4
          for (int j = 0; j < sl.y; ++j) {
            const unsigned e = __ldg(ge + 32 * j);
            s = fma(__ldg(d.pal + (e >> 20)), sm[BUF_T(d.P, e & 0xFFFFF, t)], s);
          }
        }
        sm[BUF_T(d.Gb, id, t)] = s;
      }
    }
    __syncthreads();
    if (kVar == 2 && d.digest == 5) {
      // ---- DF-J contracted at the (e 0|c) level (the analogue of a
      // J-engine: D and c meet the intermediates, not the integrals).  With
      // the pair's bra map M (HRR then bra transforms, (AB|C) = sum_e
      // M[AB][e] (e 0|C)) and the ket transform T, (e 0|C) = sum_c T[C][c] (e 0|c):
      //   gamma[t][C] = sum_c T[C][c] sum_e Dp[e] (e 0|c)_t,   Dp = w M^T D_pair
      //   y[e]       += sum_{t,c} (e 0|c)_t cp[t][c],           cp = T^T c_t
      // and J += wj M y per sub-pair once all its tiles are done
      // (jeng_finish_kernel).  No ket transform, HRR or bra transform per triple.
      const int nk = d.nkrow, ncc = d.ncc, nC = d.nC;
      double* Dp = sm + d.dscr;       // [nk]
      double* Cp = Dp + nk;           // [tv][ncc]
      double* gq = Cp + T * ncc;      // [tv][ncc]
      if (d.gacc)
        for (int e = tid; e < nk; e += kThreads) Dp[e] = __ldg(d.jD + sub * nk + e);
      if (d.Jacc)
        for (int i = tid; i < tv * ncc; i += kThreads) {
          const int t = i / ncc, c = i - t * ncc;
          const double* cv = d.cvec + __ldg(d.aux_ao + aux0 + t);
          double v = 0.0;
          for (int q = __ldg(d.ktptr + c); q < __ldg(d.ktptr + c + 1); ++q) {
            const int2 e = __ldg(d.ktent + q);
            v = fma(__ldg(d.pal + e.y), __ldg(cv + e.x), v);
          }
          Cp[i] = v;
        }
      __syncthreads();
      const Buf gb = d.Gb;
      FDiv fc;
      fc.init(ncc);
      if (d.gacc) {
        seg_dot(tv * ncc, nk,
                [&](int o, int r, double acc) {
                  const int t = (int)fc.div(o), c = o - t * ncc;
                  return fma(sm[BUF_T(gb, r * ncc + c, t)], Dp[r], acc);
                },
                [&](int o, double v) { gq[o] = v; }, true);
        __syncthreads();
        FDiv fCC;
        fCC.init(nC);
        for (int i = tid; i < tv * nC; i += kThreads) {
          const int t = (int)fCC.div(i), C = i - t * nC;
          double v = 0.0;
          for (int q = __ldg(d.kptr + C); q < __ldg(d.kptr + C + 1); ++q) {
            const int2 e = __ldg(d.kent + q);
            v = fma(__ldg(d.pal + e.y), gq[t * ncc + e.x], v);
          }
          fix_add(d.gacc + kFixWords * (__ldg(d.aux_ao + aux0 + t) + C), v);
        }
      }
      if (d.Jacc)
        seg_dot(nk, tv * ncc,
                [&](int o, int r, double acc) {
                  const int t = (int)fc.div(r), c = r - t * ncc;
                  return fma(sm[BUF_T(gb, o * ncc + c, t)], Cp[r], acc);
                },
                [&](int o, double v) { fix_add(d.jY + kFixWords * (sub * nk + o), v); });
      return;
    }
    // ---- ket: Cartesian -> solid harmonic.  With targets across lanes
    // (mode 1) the items run C-major, so a warp's lanes share one C and with
    // it the loop trip count (a warp instruction costs the same whatever the
    // number of active lanes).
    {
      FDiv fX, fC, fR;
      const int nx = d.nkrow * d.nC;
      fX.init(nx);
      fC.init(d.nC);
      fR.init(d.nkrow);
      const unsigned n = (unsigned)(T * nx);
      for (unsigned w = tid; w < n; w += kThreads) {
        int t, x;
        dec2(w, mode, fT, fX, t, x);
        if (t >= tv) continue;
        int row, C;
        if (mode == 0) {
          row = (int)fC.div(x);
          C = x - row * d.nC;
        } else {
          C = (int)fR.div(x);
          row = x - C * d.nkrow;
        }
        x = row * d.nC + C;
        const int q0 = __ldg(d.kptr + C), q1 = __ldg(d.kptr + C + 1);
        double s = 0.0;
        if (d.comp & 2) {
          Dot2 acc;
          for (int q = q0; q < q1; ++q) {
            const int2 e = __ldg(d.kent + q);
            acc.add(__ldg(d.pal + e.y), sm[BUF_T(d.Gb, row * d.ncc + e.x, t)]);
          }
          s = acc.value();
        } else {
          for (int q = q0; q < q1; ++q) {
            const int2 e = __ldg(d.kent + q);
            s = fma(__ldg(d.pal + e.y), sm[BUF_T(d.Gb, row * d.ncc + e.x, t)], s);
          }
        }
        sm[BUF_T(d.H[0], x, t)] = s;
      }
    }
    __syncthreads();
    Buf cur = hrr_and_bra(d, sm, T, tv, mode, fT);
    if (d.digest == 3) {
      // ---- matrix store (2-centre metric (P|Q) = (P 1|Q), nB = 1): element
      // (t, A, C) of the tile goes to out[(ao_pair + A) * ldD + ao_ket + C]
      const int4 pao = __ldg(d.pair_ao + pair);
      const int nA = d.onA, nC = d.nC, nAC = nA * nC;
      FDiv fAC, fC;
      fAC.init(nAC);
      fC.init(nC);
      const unsigned n = (unsigned)(tv * nAC);
      for (unsigned w = tid; w < n; w += kThreads) {
        const int t = (int)fAC.div(w), r = (int)(w - (unsigned)t * nAC);
        const int A = (int)fC.div(r), C = r - A * nC;
        d.out[(long long)(pao.x + A) * d.ldD + __ldg(d.aux_ao + aux0 + t) + C] = sm[BUF_T(cur, A * nC + C, t)];
      }
      return;
    }
    if (d.digest == 2) {
      // ---- gradient digestion: contract the derivative block with
      // W = w D_ab c_P (Cartesian in the bra) without storing it.
      const int4 pao = __ldg(d.pair_ao + pair);
      const int2 pat = __ldg(d.pair_atoms + pair);
      const double wp = pao.z ? 1.0 : 2.0;
      const int nAp = d.g_nAp, ncA = d.g_ncA, nBp = d.g_nBp, ncB = d.g_ncB, nC = d.nC, nch = d.g_nch;
      double* X = sm + d.g_base;     // [nAp][ncB]
      double* Dc = X + nAp * ncB;    // [ncA][ncB]
      double* part = Dc + ncA * ncB; // [tv][3][nch]
      for (int w = tid; w < nAp * ncB; w += kThreads) {
        const int A = w / ncB, b = w - A * ncB;
        const double* Drow = d.D + (long long)(pao.x + A) * d.ldD + pao.y;
        double s = 0.0;
        for (int B = 0; B < nBp; ++B) s = fma(__ldg(Drow + B), __ldg(d.Tb + B * ncB + b), s);
        X[w] = s;
      }
      __syncthreads();
      for (int w = tid; w < ncA * ncB; w += kThreads) {
        const int a = w / ncB, b = w - a * ncB;
        double s = 0.0;
        for (int A = 0; A < nAp; ++A) s = fma(__ldg(d.Ta + A * ncA + a), X[A * ncB + b], s);
        Dc[w] = wp * s;
      }
      __syncthreads();
      const int dnA = d.onA, dnB = d.onB;  // derivative class bra dims, caller order
      for (int w = tid; w < tv * 3 * nch; w += kThreads) {
        const int t = w / (3 * nch), rem = w - t * 3 * nch, ax = rem / nch, k = rem - ax * nch;
        const int e0 = d.gstart[ax] + k * d.g_echunk, e1 = min(d.gstart[ax + 1], e0 + d.g_echunk);
        const double* cv = d.cvec + __ldg(d.aux_ao + aux0 + t);
        double s = 0.0;
        for (int e = e0; e < e1; ++e) {
          const int4 g = __ldg(d.gmap + e);
          double tmp = 0.0;
          for (int C = 0; C < nC; ++C) {
            const int sidx = d.orient ? (g.y * dnA + g.x) * nC + C : (g.x * dnB + g.y) * nC + C;
            tmp = fma(__ldg(cv + C), sm[BUF_T(cur, sidx, t)], tmp);
          }
          s = fma((double)g.w * Dc[g.z], tmp, s);
        }
        part[w] = s;
      }
      __syncthreads();
      const int tatom = d.g_centre ? pat.y : pat.x;
      double* tsum = part + T * 3 * nch;  // [tv][3]
      for (int w = tid; w < tv * 3; w += kThreads) {
        const int t = w / 3, ax = w - t * 3;
        double s0 = 0.0, s1 = 0.0;
        int k = 0;
        for (; k + 1 < nch; k += 2) {
          s0 += part[(t * 3 + ax) * nch + k];
          s1 += part[(t * 3 + ax) * nch + k + 1];
        }
        if (k < nch) s0 += part[(t * 3 + ax) * nch + k];
        const double s = s0 + s1;
        tsum[w] = s;
        fix_add(d.facc + kFixWords * (3 * __ldg(d.aux_atom + aux0 + t) + ax), -s);
      }
      __syncthreads();
      // the pair's centre atom: the tile's kets summed first, one add per axis
      if (tid < 3) {
        double s = 0.0;
        for (int t = 0; t < tv; ++t) s += tsum[t * 3 + tid];
        fix_add(d.facc + kFixWords * (3 * tatom + tid), s);
      }
      return;
    }
    if (kVar == 1 && d.digest == 4) {
      // ---- DF-J digestion for nd <= 8 densities at once, as two small GEMMs
      // on FP64 tensor-core tiles (m8n8k4), with M rows per warp tile:
      //   gamma[d][t][C] = wg * sum_s I[t][s][C] Ds[s][d]    (M = tv*nC, K = nAB)
      //   J[d][s]        = wj * sum_{t,C} I[t][s][C] Cs[t*nC+C][d]  (M = nAB, K = tv*nC)
      const int4 pao = __ldg(d.pair_ao + pair);
      const double wg = pao.z ? 1.0 : 2.0, wj = pao.z ? 0.5 : 1.0;
      const int nA = d.onA, nB = d.onB, nC = d.nC, nAB = nA * nB, R = tv * nC, nd = d.nd;
      const int kAB = (nAB + 3) & ~3, kR = (R + 3) & ~3;
      double* Ds = sm + d.dscr;      // [kAB][8]
      double* Cs = Ds + kAB * 8;     // [kR][8]
      for (int i = tid; i < kAB * 8; i += kThreads) {
        const int r = i >> 3, dd = i & 7;  // r: storage index of (A, B)
        const int A = d.orient ? r % nA : r / nB, B = d.orient ? r / nA : r % nB;
        Ds[i] = (d.gamma && r < nAB && dd < nd)
                    ? __ldg(d.D + dd * d.dstride + (long long)(pao.x + A) * d.ldD + pao.y + B)
                    : 0.0;
      }
      for (int i = tid; i < kR * 8; i += kThreads) {
        const int r = i >> 3, dd = i & 7;
        double v = 0.0;
        if (d.J && r < R && dd < nd) {
          const int t = r / nC, C = r - t * nC;
          v = __ldg(d.cvec + dd * d.cstride + __ldg(d.aux_ao + aux0 + t) + C);
        }
        Cs[i] = v;
      }
      __syncthreads();
      const Buf cb = cur;
      const int lane = tid & 31, warp = tid >> 5, g = lane >> 2, q = lane & 3;
      constexpr int kWarps = kThreads / 32;
      if (d.gamma) {
        for (int m0 = warp * 8; m0 < R; m0 += kWarps * 8) {
          const int m = m0 + g;
          const int t = m / nC, C = m - t * nC;
          double c0 = 0.0, c1 = 0.0;
          for (int k0 = 0; k0 < kAB; k0 += 4) {
            const int k = k0 + q;
            const double a = (m < R && k < nAB) ? sm[BUF_T(cb, k * nC + C, t)] : 0.0;
            dmma_8x8x4(a, Ds[(k0 + q) * 8 + g], c0, c1);
          }
          if (m < R) {
            double* gm = d.gamma + __ldg(d.aux_ao + aux0 + t) + C;
            if (2 * q < nd) atomicAdd(gm + (2 * q) * d.cstride, wg * c0);
            if (2 * q + 1 < nd) atomicAdd(gm + (2 * q + 1) * d.cstride, wg * c1);
          }
        }
      }
      if (d.J) {
        for (int m0 = warp * 8; m0 < nAB; m0 += kWarps * 8) {
          const int m = m0 + g;  // storage index s of the block
          double c0 = 0.0, c1 = 0.0;
          for (int k0 = 0; k0 < kR; k0 += 4) {
            const int k = k0 + q;
            const int t = k / nC, C = k - t * nC;
            const double a = (m < nAB && k < R) ? sm[BUF_T(cb, m * nC + C, t)] : 0.0;
            dmma_8x8x4(a, Cs[(k0 + q) * 8 + g], c0, c1);
          }
          if (m < nAB) {
            const int A = d.orient ? m % nA : m / nB, B = d.orient ? m / nA : m % nB;
            double* Jm = d.J + (long long)(pao.x + A) * d.ldD + pao.y + B;
            if (2 * q < nd) atomicAdd(Jm + (2 * q) * d.dstride, wj * c0);
            if (2 * q + 1 < nd) atomicAdd(Jm + (2 * q + 1) * d.dstride, wj * c1);
          }
        }
      }
      return;
    }
    if (d.digest) {
      // ---- DF-J digestion (Sec. 3): the block never leaves shared memory.
      // With s the block's (A, B) index in its storage order:
      //   gamma[t][C] = wg * sum_s I[t][s][C] Ds[s]        (Ds = D block)
      //   J[s]        = wj * sum_{t,C} I[t][s][C] Cs[t][C]  (Cs = c of the tile's kets)
      const int4 pao = __ldg(d.pair_ao + pair);
      const double wg = pao.z ? 1.0 : 2.0, wj = pao.z ? 0.5 : 1.0;
      const int nA = d.onA, nB = d.onB, nC = d.nC, nAB = nA * nB;
      double* Ds = sm + d.dscr;
      double* Cs = Ds + nAB;
      const int sA = d.orient ? 1 : nB, sB = d.orient ? nA : 1;  // storage index of (A, B)
      if (d.gacc)
        for (int s = tid; s < nAB; s += kThreads) {
          const int A = s / nB, B = s - A * nB;
          Ds[A * sA + B * sB] = __ldg(d.D + (long long)(pao.x + A) * d.ldD + pao.y + B);
        }
      if (d.Jacc)
        for (int i = tid; i < tv * nC; i += kThreads) {
          const int t = i / nC, C = i - t * nC;
          Cs[i] = __ldg(d.cvec + __ldg(d.aux_ao + aux0 + t) + C);
        }
      __syncthreads();
      const Buf cb = cur;
      FDiv fC;
      fC.init(nC);
      if (d.gacc)
        seg_dot(tv * nC, nAB,
                [&](int o, int r, double acc) {
                  const int t = (int)fC.div(o), C = o - t * nC;
                  return fma(sm[BUF_T(cb, r * nC + C, t)], Ds[r], acc);
                },
                [&](int o, double v) {
                  const int t = (int)fC.div(o), C = o - t * nC;
                  fix_add(d.gacc + kFixWords * (__ldg(d.aux_ao + aux0 + t) + C), wg * v);
                });
      if (d.Jacc)
        seg_dot(nAB, tv * nC,
                [&](int o, int r, double acc) {
                  const int t = (int)fC.div(r), C = r - t * nC;
                  return fma(sm[BUF_T(cb, o * nC + C, t)], Cs[r], acc);
                },
                [&](int o, double v) {
                  const int A = d.orient ? o % nA : o / nB, B = d.orient ? o / nA : o % nB;
                  fix_add(d.Jacc + kFixWords * ((long long)(pao.x + A) * d.ldD + pao.y + B), wj * v);
                });
      return;
    }
    // ---- store the tile's contiguous output block (transposed into the
    // caller's (A, B) order for B-oriented sub-pairs; added to the block
    // already written by the A-oriented launch when the pair has both)
    {
      FDiv fB, fBC, fC;
      fB.init(d.nblk);
      fBC.init(d.onB * d.nC);
      fC.init(d.nC);
      double* o = d.out + ((pair - d.out_pair0) * d.naux + aux0) * (long long)d.nblk;
      const unsigned n = (unsigned)(tv * d.nblk);
      for (unsigned w = tid; w < n; w += kThreads) {
        const unsigned t = fB.div(w);
        const int idx = (int)(w - t * d.nblk);
        int sidx = idx;
        if (d.orient) {
          const int A = (int)fBC.div(idx), rem = idx - A * d.onB * d.nC;
          const int B = (int)fC.div(rem), C = rem - B * d.nC;
          sidx = (B * d.onA + A) * d.nC + C;
        }
        double v = sm[BUF_T(cur, sidx, (int)t)];
        if (accum) v += o[w];
        o[w] = v;
      }
    }
  }
}

// One class launch: CTAs stride over the class's tiles.
__global__ void __launch_bounds__(kThreads) eri3c_kernel(const __grid_constant__ ClassDesc d) {
  extern __shared__ double sm[];
  for (long long tile = blockIdx.x; tile < d.ntiles; tile += gridDim.x) tile_body<0>(d, tile, sm);
}

// The same for DF-J launches digesting several densities (digest == 4).
__global__ void __launch_bounds__(kThreads) eri3c_multi_kernel(const __grid_constant__ ClassDesc d) {
  extern __shared__ double sm[];
  for (long long tile = blockIdx.x; tile < d.ntiles; tile += gridDim.x) tile_body<1>(d, tile, sm);
}

// DF-J launches contracting at the (e 0|c) level (digest == 5), at the
// plain kernel's three CTAs per SM.
__global__ void __launch_bounds__(kThreads, 3) eri3c_contract_kernel(const __grid_constant__ ClassDesc d) {
  extern __shared__ double sm[];
  for (long long tile = blockIdx.x; tile < d.ntiles; tile += gridDim.x) tile_body<2>(d, tile, sm);
}

// (s s|C) classes (la = lb = 0) stored per integral, one thread per triple.
// With a = 0 the n-quantum CVRR2 has the single term u = 0, so the (0 0|c)
// target is the prerequisite P_c = sum over primitive triples of
// [00|0]^(lc) X^c (Eq. a0cv2, k = 0; X = (gamma / (gamma + zeta_c)) PC), the
// same quantities the tile kernel forms.  The NC accumulators live in
// registers and the primitive loop has no barrier; the ket transform runs
// from a shared-memory copy, and the block stores its triples' blocks
// element-major (coalesced when the triples' blocks are contiguous).
constexpr int kSsThreads = 128;

// The primitive loop of one (s s|C) triple: acc[c] += [00|0]^(lc) X^c over
// the sub-pair's primitive pairs and the ket shell's primitives.
template <int LC>
__device__ __forceinline__ void ss_prims(const ClassDesc& d, long long pair, const int4& sp, long long q,
                                         double* acc) {
  const double Cx = __ldg(d.auxc + 3 * q), Cy = __ldg(d.auxc + 3 * q + 1), Cz = __ldg(d.auxc + 3 * q + 2);
  for (int ip = 0; ip < sp.z; ++ip) {
    const double* pr = d.pairrec + (pair * d.Kab_rec + __ldg(d.primidx + sp.y + ip)) * kPairRec;
    const double gam = __ldg(pr + PR_G), K = __ldg(pr + PR_K);
    const double PCx = __ldg(pr + PR_P) - Cx, PCy = __ldg(pr + PR_P + 1) - Cy, PCz = __ldg(pr + PR_P + 2) - Cz;
    const double pc2 = fma(PCz, PCz, fma(PCy, PCy, PCx * PCx));
    for (int ic = 0; ic < d.Kc; ++ic) {
      const double zc = __ldg(d.auxrec + (q * d.Kc + ic) * kAuxRec);
      const double ccp = __ldg(d.auxrec + (q * d.Kc + ic) * kAuxRec + 1);
      const double sg = gam + zc;
      const double rs = rsqrt_fp64(sg);
      const double r = rs * rs;
      const double gr = gam * r;
      const double Tb = gam * zc * r * pc2;
      double V;
      boys_scaled(d.boys_tab, d.boys_mid, d.boys_cL, LC, LC, Tb, K * ccp * rs, &V, 0);
      if (LC == 0) {
        acc[0] += V;
      } else {
        // powers of X = gr PC; the monomials X^c in the Cartesian order (x
        // descending, then y descending), one FMA per target
        double px[LC + 1], py[LC + 1], pz[LC + 1];
        px[0] = V; py[0] = 1.0; pz[0] = 1.0;
        const double Xx = gr * PCx, Xy = gr * PCy, Xz = gr * PCz;
#pragma unroll
        for (int j = 1; j <= LC; ++j) {
          px[j] = px[j - 1] * Xx;
          py[j] = py[j - 1] * Xy;
          pz[j] = pz[j - 1] * Xz;
        }
        int c = 0;
#pragma unroll
        for (int nx = LC; nx >= 0; --nx)
#pragma unroll
          for (int ny = LC - nx; ny >= 0; --ny) {
            acc[c] = fma(px[nx], py[ny] * pz[LC - nx - ny], acc[c]);
            ++c;
          }
      }
    }
  }
}

template <int LC>
__global__ void __launch_bounds__(kSsThreads) eri3c_ss_kernel(const __grid_constant__ ClassDesc d) {
  constexpr int NC = (LC + 1) * (LC + 2) / 2, NS = 2 * LC + 1;
  __shared__ double sP[kSsThreads * (NC + 1)];
  __shared__ double sO[kSsThreads * NS];
  __shared__ long long sOff[kSsThreads];
  __shared__ int sAcc[kSsThreads];
  const int tid = threadIdx.x;
  const long long ntri = d.nsub * d.naux;
  for (long long base = (long long)blockIdx.x * kSsThreads; base < ntri; base += (long long)gridDim.x * kSsThreads) {
    const long long w = base + tid;
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    long long off = -1;
    int accum = 0;
    if (w < ntri) {
      const long long sub = w / d.naux;
      const long long q = w - sub * d.naux;
      const int4 sp = __ldg(d.subpairs + sub);
      accum = sp.w;
      off = (((long long)sp.x - d.out_pair0) * d.naux + q) * (long long)d.nblk;
      ss_prims<LC>(d, sp.x, sp, q, acc);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) sP[tid * (NC + 1) + c] = acc[c];
    sOff[tid] = off;
    sAcc[tid] = accum;
    __syncthreads();
    // ket transform: element-major over the block's triples
    for (int i = tid; i < kSsThreads * NS; i += kSsThreads) {
      const int t = i / NS, C = i - t * NS;
      double v = 0.0;
      for (int k = __ldg(d.kptr + C); k < __ldg(d.kptr + C + 1); ++k) {
        const int2 e = __ldg(d.kent + k);
        v = fma(__ldg(d.pal + e.y), sP[t * (NC + 1) + e.x], v);
      }
      sO[i] = v;
    }
    __syncthreads();
    for (int i = tid; i < kSsThreads * NS; i += kSsThreads) {
      const int t = i / NS, C = i - t * NS;
      const long long o = sOff[t];
      if (o < 0) continue;
      double v = sO[i];
      if (sAcc[t]) v += d.out[o + C];
      d.out[o + C] = v;
    }
    __syncthreads();
  }
}

// (s s|C) DF-J launches digesting per integral (digest == 1), one warp per
// tile, lanes over the tile's kets: gamma_P[C] += w D_ab (ss|P)_C per lane,
// and J_ab += w_J sum over the tile's kets and C of (ss|P)_C c_PC, reduced
// across the warp into one add.  The same sums as the tile kernel's digest.
template <int LC>
__global__ void __launch_bounds__(kSsThreads) eri3c_ss_dfj_kernel(const __grid_constant__ ClassDesc d) {
  constexpr int NC = (LC + 1) * (LC + 2) / 2, NS = 2 * LC + 1;
  __shared__ double sP[kSsThreads * (NC + 1)];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* row = sP + threadIdx.x * (NC + 1);
  const long long nwarps = (long long)gridDim.x * (kSsThreads / 32);
  for (long long tile = blockIdx.x * (long long)(kSsThreads / 32) + warp; tile < d.ntiles; tile += nwarps) {
    const int4 tt = __ldg(d.tiles + tile);
    const int4 sp = __ldg(d.subpairs + tt.x);
    const long long pair = sp.x;
    const int4 pao = __ldg(d.pair_ao + pair);
    const double wg = pao.z ? 1.0 : 2.0, wj = pao.z ? 0.5 : 1.0;
    const double Dab = d.gacc ? __ldg(d.D + (long long)pao.x * d.ldD + pao.y) : 0.0;
    double jsum = 0.0;
    for (int t0 = 0; t0 < tt.z; t0 += 32) {
      const int t = t0 + lane;
      const bool live = t < tt.z;
      double acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = 0.0;
      const long long q = tt.y + t;
      if (live) ss_prims<LC>(d, pair, sp, q, acc);
#pragma unroll
      for (int c = 0; c < NC; ++c) row[c] = acc[c];
      __syncwarp();
      if (live) {
        const int ao = __ldg(d.aux_ao + q);
#pragma unroll
        for (int C = 0; C < NS; ++C) {
          double v = 0.0;
          for (int k = __ldg(d.kptr + C); k < __ldg(d.kptr + C + 1); ++k) {
            const int2 e = __ldg(d.kent + k);
            v = fma(__ldg(d.pal + e.y), row[e.x], v);
          }
          if (d.gacc) fix_add(d.gacc + kFixWords * (ao + C), wg * Dab * v);
          if (d.Jacc) jsum = fma(v, __ldg(d.cvec + ao + C), jsum);
        }
      }
      __syncwarp();
    }
    if (d.Jacc) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) jsum += __shfl_xor_sync(0xffffffffu, jsum, o);
      if (lane == 0) fix_add(d.Jacc + kFixWords * ((long long)pao.x * d.ldD + pao.y), wj * jsum);
    }
  }
}

// (p s|C) classes, lc <= 4: la = 1, lb = 0 in the A orientation, or the
// (s p|C) class run B-oriented (recurrences on the p shell, no HRR; its
// descriptor holds the (p s|C) tables with orient = 1).  With
// a = 1_i the n-quantum CVRR2 has two terms,
//   (1_i 0|c) = (1_i 0)_{0,c} + c_i (0 0)_{1,c-1_i}    (Eq. cVRR2),
// whose prerequisites are A_i(c) = sum [1_i 0|0]^(lc) X^c and
// B(n) = sum [00|0]^(lc) Y X^n (Eq. a0cv2, Y = 1/(2(gamma+zeta_c))), with
// [1_i 0|0]^(lc) = PA_i [00|0]^(lc) - (rho/gamma) PC_i [00|0]^(lc+1)
// (Eq. vrr1): 3 ncart(lc) + ncart(lc-1) accumulators held in registers.
constexpr int kPsThreads = 64;

template <int LC>
__device__ __forceinline__ void ps_prims(const ClassDesc& d, long long pair, const int4& sp, long long q,
                                         double (&A)[3][(LC + 1) * (LC + 2) / 2], double* Bm) {
  const double Cx = __ldg(d.auxc + 3 * q), Cy = __ldg(d.auxc + 3 * q + 1), Cz = __ldg(d.auxc + 3 * q + 2);
  const int fpa = d.orient ? PR_PB : PR_PA;
  for (int ip = 0; ip < sp.z; ++ip) {
    const double* pr = d.pairrec + (pair * d.Kab_rec + __ldg(d.primidx + sp.y + ip)) * kPairRec;
    const double gam = __ldg(pr + PR_G), K = __ldg(pr + PR_K);
    const double PAx = __ldg(pr + fpa), PAy = __ldg(pr + fpa + 1), PAz = __ldg(pr + fpa + 2);
    const double PCx = __ldg(pr + PR_P) - Cx, PCy = __ldg(pr + PR_P + 1) - Cy, PCz = __ldg(pr + PR_P + 2) - Cz;
    const double pc2 = fma(PCz, PCz, fma(PCy, PCy, PCx * PCx));
    for (int ic = 0; ic < d.Kc; ++ic) {
      const double zc = __ldg(d.auxrec + (q * d.Kc + ic) * kAuxRec);
      const double ccp = __ldg(d.auxrec + (q * d.Kc + ic) * kAuxRec + 1);
      const double sg = gam + zc;
      const double rs = rsqrt_fp64(sg);
      const double r = rs * rs;
      const double gr = gam * r, rg = zc * r;
      const double Tb = gam * zc * r * pc2;
      double v2[2];
      boys_scaled(d.boys_tab, d.boys_mid, d.boys_cL, LC + 1, LC, Tb, K * ccp * rs, v2, 1);
      const double V0 = v2[0];
      const double Vx = fma(-rg * PCx, v2[1], PAx * V0), Vy = fma(-rg * PCy, v2[1], PAy * V0),
                   Vz = fma(-rg * PCz, v2[1], PAz * V0);
      double px[LC + 1], py[LC + 1], pz[LC + 1];
      px[0] = 1.0; py[0] = 1.0; pz[0] = 1.0;
      const double Xx = gr * PCx, Xy = gr * PCy, Xz = gr * PCz;
#pragma unroll
      for (int j = 1; j <= LC; ++j) {
        px[j] = px[j - 1] * Xx;
        py[j] = py[j - 1] * Xy;
        pz[j] = pz[j - 1] * Xz;
      }
      int c = 0;
#pragma unroll
      for (int nx = LC; nx >= 0; --nx)
#pragma unroll
        for (int ny = LC - nx; ny >= 0; --ny) {
          const double m = px[nx] * (py[ny] * pz[LC - nx - ny]);
          A[0][c] = fma(Vx, m, A[0][c]);
          A[1][c] = fma(Vy, m, A[1][c]);
          A[2][c] = fma(Vz, m, A[2][c]);
          ++c;
        }
      if (LC > 0) {
        const double VY = V0 * (0.5 * r);
        int n = 0;
#pragma unroll
        for (int nx = LC - 1; nx >= 0; --nx)
#pragma unroll
          for (int ny = LC - 1 - nx; ny >= 0; --ny) {
            Bm[n] = fma(VY, px[nx] * (py[ny] * pz[LC - 1 - nx - ny]), Bm[n]);
            ++n;
          }
      }
    }
  }
}

// The (p s|c) targets G(i, c) = A_i(c) + c_i B(c - 1_i) into row[i * (NC+1) + c].
template <int LC>
__device__ __forceinline__ void ps_targets(const double (&A)[3][(LC + 1) * (LC + 2) / 2], const double* Bm,
                                           double* row) {
  constexpr int NC = (LC + 1) * (LC + 2) / 2;
  int c = 0;
#pragma unroll
  for (int nx = LC; nx >= 0; --nx)
#pragma unroll
    for (int ny = LC - nx; ny >= 0; --ny) {
      const int nz = LC - nx - ny;
      // index of c - 1_i in the Cartesian order of degree LC-1
      double gx = A[0][c], gy = A[1][c], gz = A[2][c];
      if (LC > 0) {
        // position of (x, y, z) of degree LC-1: (LC-1-x)(LC-x)/2 + (LC-1-x-y)
        if (nx > 0) gx = fma((double)nx, Bm[(LC - nx) * (LC - nx + 1) / 2 + (LC - nx - ny)], gx);
        if (ny > 0) gy = fma((double)ny, Bm[(LC - 1 - nx) * (LC - nx) / 2 + (LC - nx - ny)], gy);
        if (nz > 0) gz = fma((double)nz, Bm[(LC - 1 - nx) * (LC - nx) / 2 + (LC - 1 - nx - ny)], gz);
      }
      row[c] = gx;
      row[(NC + 1) + c] = gy;
      row[2 * (NC + 1) + c] = gz;
      ++c;
    }
}

// Ket then bra transform of one triple's targets (row: 3 x (NC+1)) into
// out[s * NS + C], s the bra component in storage order.
template <int LC>
__device__ __forceinline__ void ps_transform(const ClassDesc& d, const double* row, double* out) {
  constexpr int NC = (LC + 1) * (LC + 2) / 2, NS = 2 * LC + 1;
  double H[3][NS];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int C = 0; C < NS; ++C) {
      double v = 0.0;
      for (int k = __ldg(d.kptr + C); k < __ldg(d.kptr + C + 1); ++k) {
        const int2 e = __ldg(d.kent + k);
        v = fma(__ldg(d.pal + e.y), row[a * (NC + 1) + e.x], v);
      }
      H[a][C] = v;
    }
  if (d.nbA) {
#pragma unroll
    for (int A = 0; A < 3; ++A) {
      const int q0 = __ldg(d.baptr + A), q1 = __ldg(d.baptr + A + 1);
#pragma unroll
      for (int C = 0; C < NS; ++C) {
        double v = 0.0;
        for (int k = q0; k < q1; ++k) {
          const int2 e = __ldg(d.baent + k);
          // a single 3-way select keeps H in registers
          const double h = e.x == 0 ? H[0][C] : (e.x == 1 ? H[1][C] : H[2][C]);
          v = fma(__ldg(d.pal + e.y), h, v);
        }
        out[A * NS + C] = v;
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int C = 0; C < NS; ++C) out[a * NS + C] = H[a][C];
  }
}

template <int LC>
__global__ void __launch_bounds__(kPsThreads) eri3c_ps_kernel(const __grid_constant__ ClassDesc d) {
  constexpr int NC = (LC + 1) * (LC + 2) / 2, NS = 2 * LC + 1, NB = 3 * NS;
  constexpr int NCM = LC > 0 ? LC * (LC + 1) / 2 : 1;
  __shared__ double sG[kPsThreads * 3 * (NC + 1)];
  __shared__ double sO[kPsThreads * NB];
  __shared__ long long sOff[kPsThreads];
  __shared__ int sAcc[kPsThreads];
  const int tid = threadIdx.x;
  const long long ntri = d.nsub * d.naux;
  for (long long base = (long long)blockIdx.x * kPsThreads; base < ntri; base += (long long)gridDim.x * kPsThreads) {
    const long long w = base + tid;
    long long off = -1;
    int accum = 0;
    if (w < ntri) {
      double A[3][NC], Bm[NCM];
#pragma unroll
      for (int c = 0; c < NC; ++c) A[0][c] = A[1][c] = A[2][c] = 0.0;
#pragma unroll
      for (int n = 0; n < NCM; ++n) Bm[n] = 0.0;
      const long long sub = w / d.naux;
      const long long q = w - sub * d.naux;
      const int4 sp = __ldg(d.subpairs + sub);
      accum = sp.w;
      off = (((long long)sp.x - d.out_pair0) * d.naux + q) * (long long)d.nblk;
      ps_prims<LC>(d, sp.x, sp, q, A, Bm);
      double* row = sG + tid * 3 * (NC + 1);
      ps_targets<LC>(A, Bm, row);
      ps_transform<LC>(d, row, sO + tid * NB);
    }
    sOff[tid] = off;
    sAcc[tid] = accum;
    __syncthreads();
    for (int i = tid; i < kPsThreads * NB; i += kPsThreads) {
      const int t = i / NB, x = i - t * NB;
      const long long o = sOff[t];
      if (o < 0) continue;
      double v = sO[i];
      if (sAcc[t]) v += d.out[o + x];
      d.out[o + x] = v;
    }
    __syncthreads();
  }
}

// (p s|C) DF-J launches digesting per integral: one warp per tile, lanes over
// its kets; gamma_P[C] += w sum_s D_s (ps|P)_{sC} per lane and
// J_s += w_J sum over the tile's kets and C of (ps|P)_{sC} c_PC, reduced
// across the warp.
template <int LC>
__global__ void __launch_bounds__(kPsThreads) eri3c_ps_dfj_kernel(const __grid_constant__ ClassDesc d) {
  constexpr int NC = (LC + 1) * (LC + 2) / 2, NS = 2 * LC + 1, NB = 3 * NS;
  constexpr int NCM = LC > 0 ? LC * (LC + 1) / 2 : 1;
  __shared__ double sG[kPsThreads * 3 * (NC + 1)];
  __shared__ double sO[kPsThreads * NB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* row = sG + threadIdx.x * 3 * (NC + 1);
  double* out = sO + threadIdx.x * NB;
  const long long nwarps = (long long)gridDim.x * (kPsThreads / 32);
  for (long long tile = blockIdx.x * (long long)(kPsThreads / 32) + warp; tile < d.ntiles; tile += nwarps) {
    const int4 tt = __ldg(d.tiles + tile);
    const int4 sp = __ldg(d.subpairs + tt.x);
    const long long pair = sp.x;
    const int4 pao = __ldg(d.pair_ao + pair);
    const double wg = pao.z ? 1.0 : 2.0, wj = pao.z ? 0.5 : 1.0;
    double Ds[3] = {0.0, 0.0, 0.0};
    if (d.gacc)
#pragma unroll
      for (int s = 0; s < 3; ++s)
        Ds[s] = d.orient ? __ldg(d.D + (long long)pao.x * d.ldD + pao.y + s)
                         : __ldg(d.D + (long long)(pao.x + s) * d.ldD + pao.y);
    double js[3] = {0.0, 0.0, 0.0};
    for (int t0 = 0; t0 < tt.z; t0 += 32) {
      const int t = t0 + lane;
      if (t < tt.z) {
        const long long q = tt.y + t;
        double A[3][NC], Bm[NCM];
#pragma unroll
        for (int c = 0; c < NC; ++c) A[0][c] = A[1][c] = A[2][c] = 0.0;
#pragma unroll
        for (int n = 0; n < NCM; ++n) Bm[n] = 0.0;
        ps_prims<LC>(d, pair, sp, q, A, Bm);
        ps_targets<LC>(A, Bm, row);
        ps_transform<LC>(d, row, out);
        const int ao = __ldg(d.aux_ao + q);
#pragma unroll
        for (int C = 0; C < NS; ++C) {
          const double i0 = out[C], i1 = out[NS + C], i2 = out[2 * NS + C];
          if (d.gacc) fix_add(d.gacc + kFixWords * (ao + C), wg * fma(Ds[0], i0, fma(Ds[1], i1, Ds[2] * i2)));
          if (d.Jacc) {
            const double cv = __ldg(d.cvec + ao + C);
            js[0] = fma(i0, cv, js[0]);
            js[1] = fma(i1, cv, js[1]);
            js[2] = fma(i2, cv, js[2]);
          }
        }
      }
    }
    if (d.Jacc) {
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        double v = js[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
          const long long e = d.orient ? (long long)pao.x * d.ldD + pao.y + s : (long long)(pao.x + s) * d.ldD + pao.y;
          fix_add(d.Jacc + kFixWords * e, wj * v);
        }
      }
    }
  }
}

// The bra map M of every sub-pair of a launch (digest 5): HRR and bra
// transforms applied to the unit vectors, i.e. the class stages with the nkrow
// rows of the identity in place of (e 0|C) (the descriptor has nC = nkrow,
// one "triple" per tile).  M[sub][s][e], s the block's storage index.
__global__ void __launch_bounds__(kThreads) jeng_matrix_kernel(const __grid_constant__ ClassDesc d) {
  extern __shared__ double sm[];
  const unsigned tid = threadIdx.x;
  const int nk = d.nkrow, nAB = d.onA * d.onB;
  FDiv fT;
  fT.init(1);
  for (long long sub = blockIdx.x; sub < d.nsub; sub += gridDim.x) {
    const long long pair = __ldg(d.subpairs + sub).x;
    __syncthreads();
    if (tid < 13) {
      const double sg = d.orient ? -1.0 : 1.0;
      const double x = sg * d.pairab[pair * 3], y = sg * d.pairab[pair * 3 + 1], z = sg * d.pairab[pair * 3 + 2];
      const int ax = tid >= 1 && tid <= 9 ? (int)(tid - 1) % 3 : 0;
      const double u = ax == 0 ? x : (ax == 1 ? y : z);
      double v = 1.0;
      if (tid >= 1 && tid <= 3) v = u;
      else if (tid >= 4 && tid <= 6) v = 2.0 * u;
      else if (tid >= 7 && tid <= 9) v = u * u;
      else if (tid == 10) v = x * y;
      else if (tid == 11) v = x * z;
      else if (tid == 12) v = y * z;
      sm[d.ab_base + tid] = v;
    }
    for (int w = tid; w < nk * nk; w += kThreads) sm[BUF_T(d.H[0], w, 0)] = (w / nk == w % nk) ? 1.0 : 0.0;
    __syncthreads();
    const Buf cur = hrr_and_bra(d, sm, 1, 1, 1, fT);
    double* M = d.jM + sub * (long long)nAB * nk;
    for (int w = tid; w < nAB * nk; w += kThreads) M[w] = sm[BUF_T(cur, w, 0)];
  }
}

// Dp[sub][e] = w sum_s D_s M[sub][s][e] (the pair's D block through M^T),
// one warp per sub-pair.
__global__ void jeng_dprime_kernel(const __grid_constant__ ClassDesc d) {
  const int lane = threadIdx.x & 31;
  const long long sub = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (sub >= d.nsub) return;
  const int nk = d.nkrow, nA = d.onA, nB = d.onB, nAB = nA * nB;
  const long long pair = __ldg(d.subpairs + sub).x;
  const int4 pao = __ldg(d.pair_ao + pair);
  const double w = pao.z ? 1.0 : 2.0;
  const double* M = d.jM + sub * (long long)nAB * nk;
  for (int e = lane; e < nk; e += 32) {
    double v = 0.0;
    for (int s = 0; s < nAB; ++s) {
      const int A = d.orient ? s % nA : s / nB, B = d.orient ? s / nA : s % nB;
      v = fma(__ldg(d.D + (long long)(pao.x + A) * d.ldD + pao.y + B), M[s * nk + e], v);
    }
    d.jD[sub * nk + e] = w * v;
  }
}

// J_pair += wj M y for every sub-pair (y from the fixed-point accumulators),
// one warp per sub-pair.
__global__ void jeng_finish_kernel(const __grid_constant__ ClassDesc d) {
  const int lane = threadIdx.x & 31;
  const long long sub = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (sub >= d.nsub) return;
  const int nk = d.nkrow, nA = d.onA, nB = d.onB, nAB = nA * nB;
  const long long pair = __ldg(d.subpairs + sub).x;
  const int4 pao = __ldg(d.pair_ao + pair);
  const double wj = pao.z ? 0.5 : 1.0;
  const double* M = d.jM + sub * (long long)nAB * nk;
  for (int s = lane; s < nAB; s += 32) {
    double v = 0.0;
    for (int e = 0; e < nk; ++e) v = fma(M[s * nk + e], fix_decode(d.jY + kFixWords * (sub * nk + e)), v);
    const int A = d.orient ? s % nA : s / nB, B = d.orient ? s / nA : s % nB;
    fix_add(d.Jacc + kFixWords * ((long long)(pao.x + A) * d.ldD + pao.y + B), wj * v);
  }
}

// Persistent form for mixed workloads: every CTA pulls (descriptor, tile)
// work items from one atomic counter until the list is exhausted (items are
// ordered longest first on the host).  No CTA ever waits on another.  The
// item's descriptor is staged in shared memory (re-copied only when the class
// changes), so the tile body reads its fields from there, not from global
// memory.  kMinBlocks = 3 caps the registers at 40 so that three 512-thread
// CTAs fit an SM (with a few spills to L1: the descriptor fields the
// parameter-space form keeps in constant banks now live in registers);
// kMinBlocks = 1 leaves the compiler free (64 registers, two CTAs per SM).
template <int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks) eri3c_persistent(const ClassDesc* __restrict__ descs,
                                                                         const int2* __restrict__ work, long long nwork,
                                                                         unsigned long long* __restrict__ counter) {
  extern __shared__ double sm[];
  __shared__ __align__(16) ClassDesc sd;
  __shared__ long long next;
  int cur = -1;
  constexpr int kWords = (int)(sizeof(ClassDesc) / 8);
  static_assert(sizeof(ClassDesc) % 8 == 0, "descriptor copy in 8-byte words");
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) next = (long long)atomicAdd(counter, 1ULL);
    __syncthreads();
    const long long w = next;
    if (w >= nwork) return;
    const int2 wk = work[w];
    if (wk.x != cur) {
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(descs + wk.x);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sd);
      for (int i = threadIdx.x; i < kWords; i += kThreads) dst[i] = src[i];
      cur = wk.x;
      __syncthreads();
    }
    tile_body<0>(sd, wk.y, sm);
  }
}

// Boys function evaluation for lx3c_boys: out[i*(mmax+1)+m] = F_m(T[i]).
__global__ void boys_kernel(const double* __restrict__ Tv, long long n, int mmax, const double* __restrict__ tab,
                            const double* __restrict__ mid, double cL, double* __restrict__ out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  boys_scaled(tab, mid, cL, mmax, 0, Tv[i], 1.0, out + i * (mmax + 1), 1);
}

// ---------------------------------------------------------------------------
// host-side launch helpers (called from capi.cu)
// ---------------------------------------------------------------------------

cudaError_t init_constants() {
  double v[32];
  for (int m = 0; m < 32; ++m) v[m] = 1.0 / (2 * m + 1);
  return cudaMemcpyToSymbol(c_inv2m1, v, sizeof(v));
}

cudaError_t launch_pair_precompute(const DevBasis& orb, const int32_t* pairs, long long npair, int Ka, int Kb,
                                   double* rec, double* ab, cudaStream_t st, int scale_a, int scale_b) {
  long long n = npair * Ka * Kb;
  if (n == 0) return cudaSuccess;
  pair_precompute<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(orb, pairs, npair, Ka, Kb, rec, ab, scale_a, scale_b);
  return cudaGetLastError();
}

cudaError_t launch_aux_precompute(const DevBasis& aux, const int32_t* auxs, long long naux, int Kc, double* rec,
                                  double* cxyz, cudaStream_t st) {
  long long n = naux * Kc;
  if (n == 0) return cudaSuccess;
  aux_precompute<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(aux, auxs, naux, Kc, rec, cxyz);
  return cudaGetLastError();
}

// SM count of the current device, for the grid-stride grids of the
// register-resident kernels (read once; 152 on GB300).
static int device_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 152;
    return v;
  }();
  return n;
}

cudaError_t launch_eri3c(const ClassDesc& d, int grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(eri3c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(eri3c_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(eri3c_contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (d.digest == 0 && d.la == 0 && d.lb == 0 && d.orient == 0) {
    // (s s|C): the register-resident form, one thread per triple
    const long long nb = (d.nsub * d.naux + kSsThreads - 1) / kSsThreads;
    const unsigned g = (unsigned)std::min<long long>(std::max<long long>(nb, 1), (long long)device_sms() * 32);
    switch (d.lc) {
      case 0: eri3c_ss_kernel<0><<<g, kSsThreads, 0, st>>>(d); break;
      case 1: eri3c_ss_kernel<1><<<g, kSsThreads, 0, st>>>(d); break;
      case 2: eri3c_ss_kernel<2><<<g, kSsThreads, 0, st>>>(d); break;
      case 3: eri3c_ss_kernel<3><<<g, kSsThreads, 0, st>>>(d); break;
      case 4: eri3c_ss_kernel<4><<<g, kSsThreads, 0, st>>>(d); break;
      case 5: eri3c_ss_kernel<5><<<g, kSsThreads, 0, st>>>(d); break;
      default: eri3c_ss_kernel<6><<<g, kSsThreads, 0, st>>>(d); break;
    }
  } else if ((d.digest == 0 || (d.digest == 1 && d.tiles)) && d.la == 1 && d.lb == 0 && d.lc <= 4 &&
             (d.lc > 0 || d.K > 1)) {
    // (p s|C) and B-oriented (s p|C) (whose descriptor holds the (p s|C)
    // tables with orient = 1), 1 <= lc <= 4 or contracted: register-resident.
    // (p s|s) with one primitive per triple stays on the tile kernel, which
    // measured faster there.
    const long long items = d.digest ? d.ntiles : d.nsub * d.naux;
    const long long per = d.digest ? kPsThreads / 32 : kPsThreads;
    const unsigned g = (unsigned)std::min<long long>(std::max<long long>((items + per - 1) / per, 1), (long long)device_sms() * 64);
    if (d.digest) {
      switch (d.lc) {
        case 0: eri3c_ps_dfj_kernel<0><<<g, kPsThreads, 0, st>>>(d); break;
        case 1: eri3c_ps_dfj_kernel<1><<<g, kPsThreads, 0, st>>>(d); break;
        case 2: eri3c_ps_dfj_kernel<2><<<g, kPsThreads, 0, st>>>(d); break;
        case 3: eri3c_ps_dfj_kernel<3><<<g, kPsThreads, 0, st>>>(d); break;
        default: eri3c_ps_dfj_kernel<4><<<g, kPsThreads, 0, st>>>(d); break;
      }
    } else {
      switch (d.lc) {
        case 0: eri3c_ps_kernel<0><<<g, kPsThreads, 0, st>>>(d); break;
        case 1: eri3c_ps_kernel<1><<<g, kPsThreads, 0, st>>>(d); break;
        case 2: eri3c_ps_kernel<2><<<g, kPsThreads, 0, st>>>(d); break;
        case 3: eri3c_ps_kernel<3><<<g, kPsThreads, 0, st>>>(d); break;
        default: eri3c_ps_kernel<4><<<g, kPsThreads, 0, st>>>(d); break;
      }
    }
  } else if (d.digest == 1 && d.la == 0 && d.lb == 0 && d.orient == 0 && d.tiles) {
    // (s s|C) DF-J: one warp per tile
    const long long nb = (d.ntiles + kSsThreads / 32 - 1) / (kSsThreads / 32);
    const unsigned g = (unsigned)std::min<long long>(std::max<long long>(nb, 1), (long long)device_sms() * 32);
    switch (d.lc) {
      case 0: eri3c_ss_dfj_kernel<0><<<g, kSsThreads, 0, st>>>(d); break;
      case 1: eri3c_ss_dfj_kernel<1><<<g, kSsThreads, 0, st>>>(d); break;
      case 2: eri3c_ss_dfj_kernel<2><<<g, kSsThreads, 0, st>>>(d); break;
      case 3: eri3c_ss_dfj_kernel<3><<<g, kSsThreads, 0, st>>>(d); break;
      case 4: eri3c_ss_dfj_kernel<4><<<g, kSsThreads, 0, st>>>(d); break;
      case 5: eri3c_ss_dfj_kernel<5><<<g, kSsThreads, 0, st>>>(d); break;
      default: eri3c_ss_dfj_kernel<6><<<g, kSsThreads, 0, st>>>(d); break;
    }
  } else if (d.digest == 5)
    eri3c_contract_kernel<<<grid, kThreads, (size_t)d.smem_doubles * 8, st>>>(d);
  else if (d.digest == 4)
    eri3c_multi_kernel<<<grid, kThreads, (size_t)d.smem_doubles * 8, st>>>(d);
  else
    eri3c_kernel<<<grid, kThreads, (size_t)d.smem_doubles * 8, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_jeng_matrix(const ClassDesc& d, int grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(jeng_matrix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  jeng_matrix_kernel<<<grid, kThreads, (size_t)d.smem_doubles * 8, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_jeng_pair(const ClassDesc& d, int finish, cudaStream_t st) {
  if (d.nsub == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((d.nsub + 7) / 8);
  if (finish)
    jeng_finish_kernel<<<grid, 256, 0, st>>>(d);
  else
    jeng_dprime_kernel<<<grid, 256, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_boys(const double* T, long long n, int mmax, const double* tab, const double* mid, double cL,
                        double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  boys_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(T, n, mmax, tab, mid, cL, out);
  return cudaGetLastError();
}

// The dynamic shared-memory attribute is set by persistent_occupancy(), which
// callers run before any stream capture.
cudaError_t launch_persistent(const ClassDesc* descs, const int2* work, long long nwork, unsigned long long* counter,
                              int grid, int smem_bytes, int three, cudaStream_t st) {
  if (three)
    eri3c_persistent<3><<<grid, kThreads, smem_bytes, st>>>(descs, work, nwork, counter);
  else
    eri3c_persistent<1><<<grid, kThreads, smem_bytes, st>>>(descs, work, nwork, counter);
  return cudaGetLastError();
}

int persistent_occupancy(int smem_bytes, int three) {
  int nb = 0;
  const int cap = 232448 - (int)sizeof(ClassDesc) - 64;
  cudaError_t e;
  if (three) {
    cudaFuncSetAttribute(eri3c_persistent<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eri3c_persistent<3>, kThreads, smem_bytes);
  } else {
    cudaFuncSetAttribute(eri3c_persistent<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eri3c_persistent<1>, kThreads, smem_bytes);
  }
  if (e != cudaSuccess) return 1;
  return nb < 1 ? 1 : nb;
}

int eri3c_occupancy(int smem_bytes) {
  int nb = 0;
  cudaFuncSetAttribute(eri3c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eri3c_kernel, kThreads, smem_bytes) != cudaSuccess) return 1;
  return nb < 1 ? 1 : nb;
}

}  // namespace lx3c
