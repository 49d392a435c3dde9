// Internal types shared by the host planner (plan.cu) and the device kernels
// (eri3c.cu).  Not part of the public C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <vector_types.h>
#include <vector>
#include <string>

namespace lx3c {

constexpr int kThreads = 512;            // threads per CTA of the integral kernels
constexpr int kMaxLev = 16;              // VRR1 levels (la+lb) and HRR levels (lb)
constexpr int kPairRec = 28;             // doubles per primitive-pair record
constexpr int kPairNHalf = 13;           // offset of n/(2 gamma), n = 1..14
constexpr int kAuxRec = 2;               // doubles per ket primitive record: zeta_c, c_c/zeta_c
constexpr int kBoysMmax = 24;            // Boys table covers F_0..F_24
constexpr int kBoysNF = kBoysMmax + 2;   // functions per interval: F_0..F_24, exp(-T)
constexpr int kBoysPerUnit = 8;          // intervals per unit of T (width 1/8)
constexpr int kBoysNInt = 117 * kBoysPerUnit;
constexpr double kBoysTMax = 117.0;
constexpr int kBoysDeg = 7;              // degree of the interpolating polynomial (Sec. 2.5.2)
constexpr double kDefaultAmpMax = 300.0; // orientation: largest weighted HRR amplification kept unsplit

// Pair record fields (doubles), one record per primitive pair (a_i, b_j):
//   0 gamma = za+zb
//   1 Kab'  = c_a c_b exp(-za zb/gamma |AB|^2) * 2 pi^{5/2} / gamma
//   2..4 P, 5..7 PA = P - A, 8..10 PB = P - B, 11 za, 12 zb,
//   13+n-1 = n/(2 gamma) for n = 1..14
// In shared memory a tile's records are stored in its orientation: for a
// sub-pair whose recurrences run on centre B the PB and zb fields are copied
// into the PA and za slots.
enum PairField { PR_G = 0, PR_K = 1, PR_P = 2, PR_PA = 5, PR_PB = 8, PR_ZA = 11, PR_ZB = 12, PR_NH = kPairNHalf };

// A shared-memory buffer: element (idx, g, t) lives at base + idx*si + g*sg + t*st
// (in doubles).  Per-triple buffers have sg = 0.
struct Buf {
  int base, si, sg, st;
};

// Everything a class kernel launch needs.  Passed by value (__grid_constant__).
struct ClassDesc {
  // class
  int la, lb, lc, Lab, L, bra_pure;
  int ncA, ncB, ncc;       // Cartesian sizes of the bra shells and the ket
  int nA, nB, nC, nblk;    // output block dims (nC = 2lc+1), nblk = nA*nB*nC
  int Kab, Kc, K, G, nchunk;  // Kab, K: largest sub-pair's primitive pairs, times Kc
  int Kab_rec;             // primitive-pair records per pair in pairrec (Ka*Kb)
  // orientation: 0 recurrences on A (class (la,lb)); 1 on B (class (lb,la)),
  // the block is then stored transposed into the (A, B) layout of the pair list
  int orient;
  int onA, onB;            // output block dims of the caller's (la, lb) order
  long long nsub;          // sub-pairs in this launch
  const int4* subpairs;    // {pair index, first entry in primidx, count, accumulate flag}
  const int* primidx;      // primitive-pair indices (ia*Kb + ib) of each sub-pair
  // tiling: a tile is (one sub-pair, T consecutive ket shells of the list)
  int T, Tp, mode;         // mode 0: triple index fastest across lanes; 1: target index fastest
  int ntile_aux;
  long long ntiles, npair, naux;
  // per-slot sizes
  int NV, NW, NF, NACC;
  // VRR1 levels e = 1..Lab: items [vlev_start[e-1], vlev_start[e])
  int vlev_start[kMaxLev + 1];
  int nW;                  // weight items (= NW)
  int ngt;                 // gather targets
  int nkrow;               // rows (bra Cartesian functions) entering the ket transform
  int nhrr;                // HRR rounds (lb for 1-q HRR; lb/2 + lb%2 for 2-q)
  int hrows[kMaxLev + 1];  // rows per HRR round (round 0 = nkrow)
  int hstart[kMaxLev + 1]; // first htab entry of round r (r >= 1)
  int nbA, nbB;            // bra transform output rows (A,b) and (A,B), 0 if none
  // tables (device)
  const uint4* vtab;       // VRR1 items
  const int4* wtab;        // weight items: F-buffer sources and count
  const unsigned* atab;    // accumulator -> vidx | widx<<16
  const int* gptr;         // gather CSR row pointers (by target id)
  const unsigned* gterm;   // gather terms: pidx | coef_id<<20
  // the same terms as sliced ELL for targets across lanes: slice s = targets
  // gdst[32s .. 32s+31], entry j of lane l at gell[gslice[s].x + 32 j + l]
  // (padded to the slice's longest row with zero-coefficient terms)
  const unsigned* gell;
  const int2* gslice;
  const int* gdst;         // gather item r -> target id (items sorted by term count)
  const double* pal;       // coefficient palette
  const int* kptr;         // ket CSR by C
  const int2* kent;        // (c, coef_id)
  const int* ktptr;        // the same transform transposed: CSR by c
  const int2* ktent;       // (C, coef_id)
  // HRR rows {dst | nterm << 16, src0 | src1 << 16, src2 | src3 << 16, 4-bit
  // codes of the terms' AB-product coefficients}: dst = sum_t coef_t src_t
  const uint4* htab;
  const int* baptr;        // bra A transform CSR by A: entries (a, coef_id)
  const int2* baent;
  const int* bbptr;        // bra B transform CSR by B
  const int2* bbent;
  // shared-memory layout (doubles)
  int pair_base, aux_base, ab_base;
  Buf V, W, F, P, Gb, H[kMaxLev + 1], BA, BB, OUT;
  int smem_doubles;
  // compensated (Dot2) summation in the contracted stages: bit 0 the CVRR2
  // gather, bit 1 the ket transform
  int comp;
  // data
  const double* pairrec;   // [npair][Kab][kPairRec]
  const double* pairab;    // [npair][3]  AB = A - B
  const double* auxrec;    // [naux][Kc][kAuxRec]
  const double* auxc;      // [naux][3]
  const double* boys_tab;  // [kBoysNInt][kBoysNF][8]
  const double* boys_mid;  // [kBoysNInt]
  double boys_cL;          // Gamma(L+1/2)/2 for the large-T branch
  double* out;
  long long out_pair0;     // pair index of out's first block (0 unless the output is chunked)
  // optional explicit tile table {sub-pair, first ket-list entry, ket count, 0};
  // when null, tiles are (sub-pair, T consecutive ket shells) over all naux
  const int4* tiles;
  // DF-J digestion instead of the store (Sec. 3: integral digestion callable):
  //   gamma[aux_ao[q] + C] += w * sum_AB I[A][B][C] D[ao_a + A][ao_b + B]
  //   J[ao_a + A][ao_b + B] += wj * sum_{q,C} I[A][B][C] c[aux_ao[q] + C]
  // w = 2 (1 for a == b), wj = 1 (1/2 for a == b); J is symmetrised afterwards.
  // digest == 3 stores a block with nB = 1 into the matrix out with row stride
  // ldD: out[(ao_a + A) * ldD + aux_ao[q] + C] (the 2-centre metric).
  int digest;
  int dscr;                // digestion scratch (doubles): D block [nA*nB], then c [T][nC]
  // several densities (digest == 4): nd <= 8 of them, D, cvec, gamma and J
  // holding nd matrices / vectors spaced dstride (D, J) and cstride (cvec,
  // gamma) doubles apart; the scratch holds the D blocks [nAB padded to 4][8]
  // and the tile's c values [tv*nC padded to 4][8] (zero-padded to 8 columns)
  int nd;
  long long dstride, cstride;
  // digest 1 and 2 add into exact fixed-point accumulators (fixed128.cuh),
  // two words per element, instead of the FP64 outputs: gamma [naux_ao],
  // J [nao][nao], gradient [natom][3]; NULL skips that output
  unsigned long long* gacc;
  unsigned long long* Jacc;
  unsigned long long* facc;
  // contraction at the (e 0|c) level (digest == 5, the DF-J analogue of a
  // J-engine): per sub-pair of the launch the bra map M [nAB][nkrow] (HRR and
  // bra transforms), Dp = w M^T D [nkrow] and the fixed-point y [nkrow]
  double* jM;
  double* jD;
  unsigned long long* jY;
  long long ldD;           // row stride of D and J
  const double* D;
  const double* cvec;
  double* gamma;
  double* J;
  const int4* pair_ao;     // per pair: {ao_a, ao_b, a == b, 0}
  const int* aux_ao;       // per ket-list entry: first AO
  // Gradient digestion (digest == 2): the block is a Cartesian-bra derivative
  // class ((la+-1, lb) or (la, lb+-1) in the caller's order); each entry of
  // gmap = {a', b', index into the Cartesian weight block Dc[a][b], factor}
  // adds factor * Dc[a][b] * sum_C c_C I[a'][b'][C] to dE/d(centre)_axis;
  // entries are grouped by axis (gstart[0..3]).
  int g_centre;            // 0: derivative on the pair's first shell, 1: second
  int g_nAp, g_ncA, g_nBp, g_ncB, g_nch, g_base;
  int g_echunk;            // map entries per partial sum (g_nch partials per axis)
  int gstart[4];
  const int4* gmap;
  const double* Ta;        // [2la+1][ncart(la)] of the original la
  const double* Tb;
  double* grad;            // [natom][3]
  const int2* pair_atoms;  // per pair: atoms of the two shells
  const int* aux_atom;     // per ket-list entry
};

// Device view of a basis (shell tables in HBM).
struct DevBasis {
  const int32_t* l;
  const int32_t* k;
  const int64_t* off;
  const double* xyz;
  const double* exps;
  const double* coefs;
};

// Host-side class tables (independent of the launch shape).
struct ClassTables {
  int la, lb, lc, bra_pure;
  int NV, NW, NF, NACC;
  std::vector<int> vlev_start;
  std::vector<uint4> vtab;
  std::vector<int4> wtab;
  std::vector<unsigned> atab;
  std::vector<int> gptr, gdst;
  std::vector<unsigned> gterm;
  std::vector<unsigned> gell;  // gather terms, sliced ELL (32 targets per slice, gdst order)
  std::vector<int2> gslice;    // per slice {first entry, terms per target}
  std::vector<double> pal;
  std::vector<int> kptr;
  std::vector<int2> kent;
  std::vector<int> ktptr;       // ket transform transposed (CSR by Cartesian c)
  std::vector<int2> ktent;
  int nkrow;
  int nhrr = 0, hrr2 = 0;      // HRR rounds; 1 if rounds move two quanta (Sec. 2.5.5)
  std::vector<int4> erow_xyz;  // Cartesian exponents of the nkrow round-0 rows
  std::vector<int> hrows, hstart;
  std::vector<uint4> htab;
  std::vector<int> baptr, bbptr;
  std::vector<int2> baent, bbent;
  int nbA, nbB;
  int nA, nB, nC, ncA, ncB, ncc;
  // algorithmic FP64 flop counts (FMA = 2)
  double flops_prim;      // per primitive triple
  double flops_contr;     // per contracted triple (after the primitive loop)
  // debug: (e comp, k, n comp) of each accumulator
  std::vector<int4> acc_key;
};

// Device-side constant tables (capi.cu)
struct DevClass {
  void* blob = nullptr;
  const uint4* vtab;
  const int4* wtab;
  const unsigned* atab;
  const int* gptr;
  const unsigned* gterm;
  const unsigned* gell;
  const int2* gslice;
  const int* gdst;
  const double* pal;
  const int* kptr;
  const int2* kent;
  const int* ktptr;
  const int2* ktent;
  const uint4* htab;
  const int* baptr;
  const int2* baent;
  const int* bbptr;
  const int2* bbent;
};
struct DevState;
int device_state_get(DevState** out);                       // lx3c_status
int device_class_get(DevState* s, const ClassTables& ct, DevClass** out);
const double* dev_boys_tab(const DevState* s);
const double* dev_boys_mid(const DevState* s);
int dev_nsm(const DevState* s);
int dev_smem(const DevState* s);
void set_last_error(const std::string& msg);
// Fill a launch descriptor for class (l1 l2|lc) (orientation `orient` of the
// caller's (la, lb)), kmax primitive pairs per sub-pair; returns smem bytes or
// -1 if the class does not fit.
int fill_class_desc(ClassDesc& d, const ClassTables& ct, const DevClass& dc, const DevState* ds, int orient,
                    int kmax, int Kab_rec, int Kc, long long naux_for_shape);
struct LaunchShape;
// The shape-independent part of that fill plus the layout for shape sh, with
// the class tables at dc and the Boys table at boys_tab / boys_mid (shared by
// the planned and the allocation-free paths).
void fill_desc_common(ClassDesc& d, const ClassTables& ct, const DevClass& dc, const double* boys_tab,
                      const double* boys_mid, int orient, int kmax, int Kab_rec, int Kc, const LaunchShape& sh);
// Device pointers of every class table inside one uploaded blob laid out by
// class_blob (same offsets on host and device).
std::vector<char> class_blob(const ClassTables& ct, size_t offs[18]);
void class_blob_pointers(DevClass& dc, const void* dev_blob, const size_t offs[18]);

// planner entry points (plan.cu)
const ClassTables& class_tables(int la, int lb, int lc, int bra_pure);  // HRR variant from the hints
const ClassTables& class_tables_variant(int la, int lb, int lc, int bra_pure, int hrr2);
void set_hrr_hint(int la, int lb, int lc, int bra_pure, int variant);  // variant < 0 removes the hint
int hrr_variant(int la, int lb, int lc, int bra_pure);
std::vector<double> solid_matrix(int l);   // [(m+l)*ncart(l) + c]
int ncart(int l);
int cart_index(int x, int y, int z);       // index of (x,y,z) within its shell
// Boys tables (boys.cu)
void boys_tables(std::vector<double>& tab, std::vector<double>& mid);
long double boys_ref(int m, long double T);
double boys_large_const(int L);

// Launch-shape choice and descriptor fill (plan.cu)
struct LaunchShape {
  int T, G, mode;
  int smem_bytes;
};
// Places the DF-J digestion scratch (D block and the tile's c values) in the
// stage region the final block does not occupy, or appends it when that region
// is too small; updates d.dscr and d.smem_doubles.
void set_digest_scratch(ClassDesc& d);
// Base (doubles) of `need` doubles of epilogue scratch: the stage region the
// final block does not occupy when it is large enough, else appended (grows
// d.smem_doubles).
int place_epilogue_scratch(ClassDesc& d, long long need);
std::string check_class_tables(const ClassTables& ct);  // "" when every table invariant holds
// Largest relative error of the class's HRR tables applied to moment
// integrals (exact for any weight), see lx3c_hrr_tables_check.
double hrr_moment_error(const ClassTables& ct, const double AB[3]);
LaunchShape choose_shape(const ClassTables& ct, int Kab, int Kc, long long naux, int smem_limit);
LaunchShape choose_shape_for(const ClassTables& ct, int Kab, int Kc, long long naux, int smem_limit, int ctas);
void set_shape_hint(int la, int lb, int lc, int bra_pure, int Kab, int Kc, int ctas);
void set_tile_hint(int la, int lb, int lc, int bra_pure, int Kab, int Kc, int T, int G);
void fill_layout(ClassDesc& d, const ClassTables& ct, const LaunchShape& s);

// Process-wide accuracy settings (capi.cu): the orientation split's
// amplification threshold and the compensated-summation bits of new plans.
double orientation_amp_max();
int compensation_bits();
}  // namespace lx3c

// Shell table, host copy plus device SoA copy (opaque in the C ABI).
struct lx3c_basis {
  int64_t nshell = 0, nprim = 0;
  std::vector<int32_t> l, k, atom;
  std::vector<int64_t> off;
  std::vector<double> xyz, exps, coefs;
  int32_t* d_l = nullptr;
  int32_t* d_k = nullptr;
  int64_t* d_off = nullptr;
  double* d_xyz = nullptr;
  double* d_exps = nullptr;
  double* d_coefs = nullptr;
  lx3c::DevBasis dev() const { return lx3c::DevBasis{d_l, d_k, d_off, d_xyz, d_exps, d_coefs}; }
};

namespace lx3c {
// Allocate and fill the device copy of a basis from its host vectors
// (synchronises st).  No validation: callers check the shell table first.
int basis_upload(lx3c_basis* b, cudaStream_t st);
// Orientation of a pair: its primitive pairs go to primA or primB -- all to
// the orientation with the smaller weighted HRR amplification when that is
// at most the orientation threshold, else each to its more compact centre.
void split_orientation(const lx3c_basis* orb, int a, int b, int la, int lb, std::vector<int>& primA,
                       std::vector<int>& primB);
}  // namespace lx3c
