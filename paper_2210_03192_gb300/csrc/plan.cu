// Host-side class planner: builds, once per (la, lb | lc, bra_pure), the index
// tables that drive the integral kernel's stages, and chooses the launch shape.
//
// Stages and the passages they follow (arXiv:2210.03192):
//   [00|0]^(m)       Sec. 2.5.2 (Boys function times the prefactor)
//   VRR1             Eq. vrr1: [a+1_i 0|0]^(m) = PA_i [a]^(m) - rho/gamma PC_i [a]^(m+1)
//                              + a_i/(2 gamma) ([a-1_i]^(m) - rho/gamma [a-1_i]^(m+1))
//   CVRR2 prerequisites  Eq. a0cv2: (e 0)_{k,n} = sum_prim Y^k X^n [e 0|0]^(lc),
//                    Y = rho/(2 gamma zeta_c) = 1/(2(gamma+zeta_c)), X = rho/zeta_c PC
//   CVRR2 targets    n-q form of Eq. cVRR2 (the printed closed form is garbled; the
//                    reading used is sum over u <= min(a,c) of
//                    prod_i C(a_i,u_i) C(c_i,u_i) u_i! (a-u 0)_{|u|, c-u})
//   ket transform    Sec. 2.5.1 (Cartesian ket to solid harmonic)
//   HRR              Eq. hrr: (a b+1_i|C) = (a+1_i b|C) + AB_i (a b|C)
//   bra transform    optional (solid-harmonic bra)
#include <vector_types.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <map>
#include <mutex>
#include <set>
#include <stdexcept>
#include <string>
#include <tuple>

#include "lx3c_internal.h"

namespace lx3c {

int ncart(int l) { return l < 0 ? 0 : (l + 1) * (l + 2) / 2; }

int cart_index(int x, int y, int z) {
  int l = x + y + z, idx = 0;
  for (int ax = l; ax > x; --ax) idx += l - ax + 1;
  return idx + (l - x) - y;
}

namespace {

struct C3 {
  int v[3];
  int l() const { return v[0] + v[1] + v[2]; }
  bool operator<(const C3& o) const { return std::tie(v[0], v[1], v[2]) < std::tie(o.v[0], o.v[1], o.v[2]); }
  bool operator==(const C3& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2]; }
};

std::vector<C3> cart(int l) {
  std::vector<C3> out;
  for (int x = l; x >= 0; --x)
    for (int y = l - x; y >= 0; --y) out.push_back(C3{{x, y, l - x - y}});
  return out;
}

double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return std::round(r);
}

double fact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

}  // namespace

// Real solid harmonics, Racah normalisation, m = -l..l, by the closed
// expansion of S_lm in Cartesian monomials (standard Schlegel-Frisch /
// Helgaker form): S_lm = N_lm sum_{t,u,v} C_tuv x^{2t+|m|-2(u+v)} y^{2(u+v)} z^{l-2t-|m|}.
std::vector<double> solid_matrix(int l) {
  int nc = ncart(l);
  std::vector<double> T((2 * l + 1) * nc, 0.0);
  for (int m = -l; m <= l; ++m) {
    int am = m < 0 ? -m : m;
    int vm2 = m < 0 ? 1 : 0;  // 2*v_m
    long double N = 1.0L / (std::pow(2.0L, am) * (long double)fact(l)) *
                    std::sqrt(2.0L * (long double)fact(l + am) * (long double)fact(l - am) / (m == 0 ? 2.0L : 1.0L));
    for (int t = 0; t <= (l - am) / 2; ++t)
      for (int u = 0; u <= t; ++u)
        for (int vv = vm2; vv <= am; vv += 2) {  // vv = 2v
          int sgn_exp = t + (vv - vm2) / 2;
          long double c = ((sgn_exp & 1) ? -1.0L : 1.0L) * std::pow(0.25L, t) * binom(l, t) * binom(l - t, am + t) *
                          binom(t, u) * binom(am, vv);
          int ex = 2 * t + am - 2 * u - vv, ey = 2 * u + vv, ez = l - 2 * t - am;
          if (ex < 0) continue;
          T[(m + l) * nc + cart_index(ex, ey, ez)] += (double)(N * c);
        }
  }
  return T;
}

namespace {

unsigned pal_id(std::vector<double>& pal, std::map<double, int>& ids, double v) {
  auto it = ids.find(v);
  if (it != ids.end()) return it->second;
  int id = (int)pal.size();
  pal.push_back(v);
  ids[v] = id;
  return id;
}

ClassTables build(int la, int lb, int lc, int bra_pure, int hrr2) {
  ClassTables ct;
  ct.la = la; ct.lb = lb; ct.lc = lc; ct.bra_pure = bra_pure;
  const int Lab = la + lb;
  ct.ncA = ncart(la); ct.ncB = ncart(lb); ct.ncc = ncart(lc);
  ct.nC = 2 * lc + 1;
  ct.nA = bra_pure ? 2 * la + 1 : ct.ncA;
  ct.nB = bra_pure ? 2 * lb + 1 : ct.ncB;
  std::map<double, int> palids;
  pal_id(ct.pal, palids, 1.0);  // id 0 is always 1.0

  // ---------------- HRR dependency analysis (Eq. hrr) ----------------
  // Rounds r = 1..R move q_r quanta from the recurrence centre to the other:
  // every q_r = 1 (1-q HRR, Eq. hrr), or with hrr2 the 2-quantum transfer of
  // Sec. 2.5.5 applied twice in one round,
  //   (a, b+1_i+1_k) = (a+1_i+1_k, b) + AB_i (a+1_k, b) + AB_k (a+1_i, b) + AB_i AB_k (a, b),
  // with one 1-q round last (topmost) when lb is odd.  Nodes (a, b) of round
  // r have |b| = the quanta moved so far; the top round holds every (a, b) of
  // the target, and each round keeps only the nodes the next one reads
  // (greedy cover: as few lower b's as possible).
  std::vector<int> step;  // q_r, r = 1..R, bottom-up
  if (hrr2) {
    for (int q = 0; q < lb / 2; ++q) step.push_back(2);
    if (lb & 1) step.push_back(1);
  } else {
    for (int q = 0; q < lb; ++q) step.push_back(1);
  }
  const int R = (int)step.size();
  std::vector<int> bl(R + 1, 0);  // |b| of round r
  for (int r = 1; r <= R; ++r) bl[r] = bl[r - 1] + step[r - 1];
  std::vector<std::vector<std::pair<C3, C3>>> lev(R + 1);
  std::vector<std::map<std::pair<C3, C3>, int>> levidx(R + 1);
  // per needed b of round r: the lower b and the axes (i, k) (k = -1 for 1-q)
  std::vector<std::map<C3, std::pair<C3, std::pair<int, int>>>> bdec(R + 1);
  for (auto& a : cart(la))
    for (auto& b : cart(lb)) {
      levidx[R][{a, b}] = (int)lev[R].size();
      lev[R].push_back({a, b});
    }
  auto add = [](C3 x, int i, int k) {
    if (i >= 0) x.v[i]++;
    if (k >= 0) x.v[k]++;
    return x;
  };
  for (int r = R; r >= 1; --r) {
    const int q = step[r - 1];
    std::set<C3> need;
    for (auto& n : lev[r]) need.insert(n.second);
    while (!need.empty()) {
      C3 best{{0, 0, 0}};
      int bestcount = -1;
      for (auto& bp : cart(bl[r - 1])) {
        int cnt = 0;
        for (int i = 0; i < 3; ++i)
          for (int k = (q == 2 ? i : -1); k < (q == 2 ? 3 : 0); ++k)
            if (need.count(add(bp, i, k))) ++cnt;
        if (cnt > bestcount) { bestcount = cnt; best = bp; }
      }
      for (int i = 0; i < 3; ++i)
        for (int k = (q == 2 ? i : -1); k < (q == 2 ? 3 : 0); ++k) {
          C3 b = add(best, i, k);
          if (need.count(b)) { bdec[r][b] = {best, {i, k}}; need.erase(b); }
        }
    }
    std::set<std::pair<C3, C3>> prev;
    for (auto& n : lev[r]) {
      const auto& dec = bdec[r][n.second];
      const C3& bp = dec.first;
      const int i = dec.second.first, k = dec.second.second;
      prev.insert({add(n.first, i, k), bp});
      prev.insert({n.first, bp});
      if (k >= 0) {
        prev.insert({add(n.first, i, -1), bp});
        prev.insert({add(n.first, k, -1), bp});
      }
    }
    // order the lower round's nodes: by |a|, then a, then b
    std::vector<std::pair<C3, C3>> pv(prev.begin(), prev.end());
    std::sort(pv.begin(), pv.end(), [](const std::pair<C3, C3>& x, const std::pair<C3, C3>& y) {
      if (x.first.l() != y.first.l()) return x.first.l() < y.first.l();
      int ix = cart_index(x.first.v[0], x.first.v[1], x.first.v[2]);
      int iy = cart_index(y.first.v[0], y.first.v[1], y.first.v[2]);
      if (ix != iy) return ix < iy;
      return cart_index(x.second.v[0], x.second.v[1], x.second.v[2]) <
             cart_index(y.second.v[0], y.second.v[1], y.second.v[2]);
    });
    lev[r - 1] = pv;
    for (size_t n = 0; n < pv.size(); ++n) levidx[r - 1][pv[n]] = (int)n;
  }
  // e0 rows (round 0): needed bra functions (a, 0)
  std::vector<C3> erows;
  for (auto& n : lev[0]) erows.push_back(n.first);
  ct.nkrow = (int)erows.size();
  for (auto& e : erows) ct.erow_xyz.push_back(int4{e.v[0], e.v[1], e.v[2], 0});
  ct.nhrr = R;
  ct.hrr2 = hrr2;
  ct.hrows.assign(R + 1, 0);
  ct.hstart.assign(R + 2, 0);
  ct.hrows[0] = ct.nkrow;
  // row = {dst | nterm << 16, src0 | src1 << 16, src2 | src3 << 16, 4-bit
  // coefficient codes}; codes index the tile's AB products: 0 one, 1..3 AB_i,
  // 4..6 2 AB_i, 7..9 AB_i^2, 10 AB_x AB_y, 11 AB_x AB_z, 12 AB_y AB_z
  auto pcode = [](int i, int k) {
    if (i == k) return 7 + i;
    const int lo = std::min(i, k), hi = std::max(i, k);
    return lo == 0 ? (hi == 1 ? 10 : 11) : 12;
  };
  for (int r = 1; r <= R; ++r) {
    ct.hstart[r] = (int)ct.htab.size();
    ct.hrows[r] = (int)lev[r].size();
    std::vector<std::pair<int, uint4>> rows;
    for (size_t n = 0; n < lev[r].size(); ++n) {
      const auto& node = lev[r][n];
      const auto& dec = bdec[r][node.second];
      const C3& bp = dec.first;
      const int i = dec.second.first, k = dec.second.second;
      const C3& a = node.first;
      unsigned src[4] = {0, 0, 0, 0}, code[4] = {0, 0, 0, 0};
      int nt;
      auto at = [&](const C3& x) { return (unsigned)levidx[r - 1].at({x, bp}); };
      if (k < 0) {
        src[0] = at(add(a, i, -1)); code[0] = 0;
        src[1] = at(a); code[1] = 1 + i;
        nt = 2;
      } else if (i == k) {
        src[0] = at(add(a, i, i)); code[0] = 0;
        src[1] = at(add(a, i, -1)); code[1] = 4 + i;
        src[2] = at(a); code[2] = pcode(i, i);
        nt = 3;
      } else {
        src[0] = at(add(a, i, k)); code[0] = 0;
        src[1] = at(add(a, k, -1)); code[1] = 1 + i;
        src[2] = at(add(a, i, -1)); code[2] = 1 + k;
        src[3] = at(a); code[3] = pcode(i, k);
        nt = 4;
      }
      rows.push_back({nt, uint4{(unsigned)n | ((unsigned)nt << 16), src[0] | (src[1] << 16), src[2] | (src[3] << 16),
                                code[0] | (code[1] << 4) | (code[2] << 8) | (code[3] << 12)}});
    }
    // rows with the same term count together, so that a warp's lanes share it
    std::stable_sort(rows.begin(), rows.end(), [](auto& x, auto& y) { return x.first < y.first; });
    for (auto& rw : rows) ct.htab.push_back(rw.second);
  }
  ct.hstart[R + 1] = (int)ct.htab.size();

  // ---------------- VRR1 buffer and items (Eq. vrr1) ----------------
  std::vector<int> voff(Lab + 2, 0);
  for (int e = 0; e <= Lab; ++e) voff[e + 1] = voff[e] + ncart(e) * (Lab - e + 1);
  ct.NV = voff[Lab + 1];
  auto vidx = [&](int e, int m, const C3& c) { return voff[e] + (m - lc) * ncart(e) + cart_index(c.v[0], c.v[1], c.v[2]); };
  ct.vlev_start.assign(Lab + 1, 0);
  for (int e = 1; e <= Lab; ++e) {
    ct.vlev_start[e - 1] = (int)ct.vtab.size();
    std::vector<uint4> simple, full;
    for (auto& t : cart(e)) {
      int ax = -1;
      for (int i = 0; i < 3; ++i)
        if (t.v[i] == 1) { ax = i; break; }
      if (ax < 0)
        for (int i = 0; i < 3; ++i)
          if (t.v[i] > 0 && (ax < 0 || t.v[i] > t.v[ax])) ax = i;
      int n = t.v[ax] - 1;
      C3 s1 = t;
      s1.v[ax]--;
      C3 s2 = s1;
      if (n > 0) s2.v[ax]--;
      for (int m = lc; m <= lc + Lab - e; ++m) {
        unsigned dst = vidx(e, m, t), a = vidx(e - 1, m, s1), an = vidx(e - 1, m + 1, s1);
        unsigned b = n > 0 ? vidx(e - 2, m, s2) : 0u, bn = n > 0 ? vidx(e - 2, m + 1, s2) : 0u;
        uint4 it{dst | (a << 16), an | (b << 16), bn | ((unsigned)ax << 16) | ((unsigned)n << 20), 0u};
        (n > 0 ? full : simple).push_back(it);
      }
    }
    ct.vtab.insert(ct.vtab.end(), simple.begin(), simple.end());
    ct.vtab.insert(ct.vtab.end(), full.begin(), full.end());
  }
  ct.vlev_start[Lab] = (int)ct.vtab.size();

  // ---------------- weights W_{k,n} = Y^k X^n (Eq. a0cv2) ----------------
  // F buffer: 0..2 (rho/gamma) PC, 3 rho/gamma, 4 + i*lc + (j-1) X_i^j, 4 + 3lc + (k-1) Y^k
  ct.NF = 4 + 4 * lc;
  std::vector<int> woff(lc + 2, 0);
  for (int k = 0; k <= lc; ++k) woff[k + 1] = woff[k] + ncart(lc - k);
  ct.NW = woff[lc + 1];
  {
    std::vector<std::pair<int, int4>> items;
    for (int k = 0; k <= lc; ++k)
      for (auto& n : cart(lc - k)) {
        int w = woff[k] + cart_index(n.v[0], n.v[1], n.v[2]);
        std::vector<int> src;
        if (k > 0) src.push_back(4 + 3 * lc + (k - 1));
        for (int i = 0; i < 3; ++i)
          if (n.v[i] > 0) src.push_back(4 + i * lc + (n.v[i] - 1));
        while (src.size() < 4) src.push_back(0xFFFF);
        int cnt = 0;
        for (int s : src) cnt += s != 0xFFFF;
        int4 it{w | (src[0] << 16), src[1] | (src[2] << 16), src[3] | (cnt << 16), 0};
        items.push_back({cnt, it});
      }
    std::stable_sort(items.begin(), items.end(), [](auto& x, auto& y) { return x.first < y.first; });
    for (auto& it : items) ct.wtab.push_back(it.second);
  }

  // ---------------- CVRR2 targets and prerequisites (Sec. 2.5.4) ----------------
  std::map<std::tuple<C3, int, C3>, int> accmap;
  std::vector<std::tuple<C3, int, C3>> acckeys;
  auto cl = cart(lc);
  struct Tgt { int id; std::vector<unsigned> terms; };
  std::vector<Tgt> tg;
  std::vector<std::vector<std::pair<std::tuple<C3, int, C3>, double>>> rawterms;
  for (int r = 0; r < ct.nkrow; ++r) {
    const C3& a = erows[r];
    for (size_t ic = 0; ic < cl.size(); ++ic) {
      const C3& c = cl[ic];
      std::vector<std::pair<std::tuple<C3, int, C3>, double>> terms;
      for (int ux = 0; ux <= std::min(a.v[0], c.v[0]); ++ux)
        for (int uy = 0; uy <= std::min(a.v[1], c.v[1]); ++uy)
          for (int uz = 0; uz <= std::min(a.v[2], c.v[2]); ++uz) {
            int u[3] = {ux, uy, uz};
            double coef = 1.0;
            C3 e, n;
            for (int i = 0; i < 3; ++i) {
              coef *= binom(a.v[i], u[i]) * binom(c.v[i], u[i]) * fact(u[i]);
              e.v[i] = a.v[i] - u[i];
              n.v[i] = c.v[i] - u[i];
            }
            terms.push_back({std::make_tuple(e, ux + uy + uz, n), coef});
          }
      rawterms.push_back(terms);
      for (auto& t : terms)
        if (!accmap.count(t.first)) { accmap[t.first] = 0; }
    }
  }
  // accumulator order: by |e|, e, k, n
  for (auto& kv : accmap) acckeys.push_back(kv.first);
  std::sort(acckeys.begin(), acckeys.end(), [](auto& x, auto& y) {
    const C3 &ex = std::get<0>(x), &ey = std::get<0>(y);
    if (ex.l() != ey.l()) return ex.l() < ey.l();
    int ix = cart_index(ex.v[0], ex.v[1], ex.v[2]), iy = cart_index(ey.v[0], ey.v[1], ey.v[2]);
    if (ix != iy) return ix < iy;
    if (std::get<1>(x) != std::get<1>(y)) return std::get<1>(x) < std::get<1>(y);
    const C3 &nx = std::get<2>(x), &ny = std::get<2>(y);
    return cart_index(nx.v[0], nx.v[1], nx.v[2]) < cart_index(ny.v[0], ny.v[1], ny.v[2]);
  });
  for (size_t i = 0; i < acckeys.size(); ++i) accmap[acckeys[i]] = (int)i;
  ct.NACC = (int)acckeys.size();
  for (auto& key : acckeys) {
    const C3& e = std::get<0>(key);
    int k = std::get<1>(key);
    const C3& n = std::get<2>(key);
    unsigned v = vidx(e.l(), lc, e);
    unsigned w = woff[k] + cart_index(n.v[0], n.v[1], n.v[2]);
    ct.atab.push_back(v | (w << 16));
    ct.acc_key.push_back(int4{cart_index(e.v[0], e.v[1], e.v[2]) | (e.l() << 16), k,
                              cart_index(n.v[0], n.v[1], n.v[2]) | ((lc - k) << 16), 0});
  }
  {
    // keep only the weights some accumulator reads (for la + lb < lc the
    // targets reach k <= la + lb only) and renumber them densely
    std::vector<int> remap(ct.NW, -1);
    for (unsigned a : ct.atab) remap[a >> 16] = 0;
    std::vector<int4> kept;
    for (const int4& it : ct.wtab) {
      const int dst = it.x & 0xFFFF;
      if (remap[dst] < 0) continue;
      remap[dst] = (int)kept.size();
      int4 k2 = it;
      k2.x = (it.x & ~0xFFFF) | remap[dst];
      kept.push_back(k2);
    }
    for (unsigned& a : ct.atab) a = (a & 0xFFFF) | ((unsigned)remap[a >> 16] << 16);
    ct.wtab = kept;
    ct.NW = (int)kept.size();
  }
  // gather CSR by target id = row*ncc + c, items sorted by descending term count
  int ngt = ct.nkrow * ct.ncc;
  ct.gptr.assign(ngt + 1, 0);
  for (int id = 0; id < ngt; ++id) {
    for (auto& t : rawterms[id]) {
      unsigned pid = (unsigned)accmap[t.first];
      unsigned cid = pal_id(ct.pal, palids, t.second);
      ct.gterm.push_back(pid | (cid << 20));
    }
    ct.gptr[id + 1] = (int)ct.gterm.size();
  }
  ct.gdst.resize(ngt);
  for (int i = 0; i < ngt; ++i) ct.gdst[i] = i;
  std::stable_sort(ct.gdst.begin(), ct.gdst.end(), [&](int x, int y) {
    return (ct.gptr[x + 1] - ct.gptr[x]) > (ct.gptr[y + 1] - ct.gptr[y]);
  });
  {
    // sliced ELL copy: padding terms read accumulator 0 with coefficient 0
    const unsigned pad = 0u | (pal_id(ct.pal, palids, 0.0) << 20);
    for (int s0 = 0; s0 < ngt; s0 += 32) {
      int mx = 0;
      for (int l = s0; l < std::min(ngt, s0 + 32); ++l) mx = std::max(mx, ct.gptr[ct.gdst[l] + 1] - ct.gptr[ct.gdst[l]]);
      ct.gslice.push_back(int2{(int)ct.gell.size(), mx});
      for (int j = 0; j < mx; ++j)
        for (int l = 0; l < 32; ++l) {
          const int r = s0 + l;
          const int id = r < ngt ? ct.gdst[r] : -1;
          const bool has = id >= 0 && j < ct.gptr[id + 1] - ct.gptr[id];
          ct.gell.push_back(has ? ct.gterm[ct.gptr[id] + j] : pad);
        }
    }
  }

  // ---------------- ket transform ----------------
  auto Tc = solid_matrix(lc);
  ct.kptr.assign(ct.nC + 1, 0);
  for (int C = 0; C < ct.nC; ++C) {
    for (int c = 0; c < ct.ncc; ++c) {
      double v = Tc[C * ct.ncc + c];
      if (v != 0.0) ct.kent.push_back(int2{c, (int)pal_id(ct.pal, palids, v)});
    }
    ct.kptr[C + 1] = (int)ct.kent.size();
  }
  ct.ktptr.assign(ct.ncc + 1, 0);
  for (int c = 0; c < ct.ncc; ++c) {
    for (int C = 0; C < ct.nC; ++C) {
      double v = Tc[C * ct.ncc + c];
      if (v != 0.0) ct.ktent.push_back(int2{C, (int)pal_id(ct.pal, palids, v)});
    }
    ct.ktptr[c + 1] = (int)ct.ktent.size();
  }

  // ---------------- bra transforms ----------------
  ct.nbA = ct.nbB = 0;
  if (bra_pure && la > 0) {
    auto Ta = solid_matrix(la);
    ct.baptr.assign(2 * la + 2, 0);
    for (int A = 0; A < 2 * la + 1; ++A) {
      for (int a = 0; a < ct.ncA; ++a) {
        double v = Ta[A * ct.ncA + a];
        if (v != 0.0) ct.baent.push_back(int2{a, (int)pal_id(ct.pal, palids, v)});
      }
      ct.baptr[A + 1] = (int)ct.baent.size();
    }
    ct.nbA = (2 * la + 1) * ct.ncB;
  }
  if (bra_pure && lb > 0) {
    auto Tb = solid_matrix(lb);
    ct.bbptr.assign(2 * lb + 2, 0);
    for (int B = 0; B < 2 * lb + 1; ++B) {
      for (int b = 0; b < ct.ncB; ++b) {
        double v = Tb[B * ct.ncB + b];
        if (v != 0.0) ct.bbent.push_back(int2{b, (int)pal_id(ct.pal, palids, v)});
      }
      ct.bbptr[B + 1] = (int)ct.bbent.size();
    }
    ct.nbB = ct.nA * (2 * lb + 1);
  }
  if (ct.pal.size() >= 4096) throw std::runtime_error("coefficient palette overflow");
  if (ct.NACC >= (1 << 20) || ct.NV >= 65536 || ct.NW >= 65536) throw std::runtime_error("class too large");

  // ---------------- algorithmic flop counts (FMA = 2) ----------------
  double fp = 0;
  // geometry, rsqrt, prefactor, factor powers ((rho/gamma) PC only when VRR1 runs)
  fp += 32 + (lc > 0 ? 4.0 * (lc - 1) : 0.0) - (Lab == 0 ? 3.0 : 0.0);
  // Boys and [00|0]^(m): one degree-7 polynomial for F_L; the exp(-T)
  // polynomial and the downward relation only when Lab > 0 (F_L..F_lc)
  fp += Lab == 0 ? 16.0 : 32.0 + 3.0 * Lab;
  for (int e = 1; e <= Lab; ++e)
    for (int i = ct.vlev_start[e - 1]; i < ct.vlev_start[e]; ++i) fp += ((ct.vtab[i].z >> 20) & 0xF) ? 7 : 3;
  for (auto& w : ct.wtab) {
    int cnt = (w.z >> 16) & 0xFFFF;
    fp += cnt > 1 ? cnt - 1 : 0;
  }
  fp += 2.0 * ct.NACC;
  ct.flops_prim = fp;
  double fc = 2.0 * ct.gterm.size();
  fc += 2.0 * ct.kent.size() * ct.nkrow;
  for (const uint4& h : ct.htab) fc += 2.0 * ((h.x >> 16) - 1) * ct.nC;
  auto bra = [&](const std::vector<int>& ptr, const std::vector<int2>& ent, int nother) {
    double f = 0;
    for (size_t A = 0; A + 1 < ptr.size(); ++A) {
      int n = ptr[A + 1] - ptr[A];
      bool copy = (n == 1 && ct.pal[ent[ptr[A]].y] == 1.0);
      if (!copy) f += 2.0 * n;
    }
    return f * nother * ct.nC;
  };
  if (ct.nbA) fc += bra(ct.baptr, ct.baent, ct.ncB);
  if (ct.nbB) fc += bra(ct.bbptr, ct.bbent, ct.nA);
  ct.flops_contr = fc;
  return ct;
}

}  // namespace

namespace {
std::mutex g_hrr_mu;
std::map<std::tuple<int, int, int, int>, int> g_hrr_hints;  // (la, lb, lc, pure) -> 0: 1-q, 1: 2-q HRR
}  // namespace

void set_hrr_hint(int la, int lb, int lc, int bra_pure, int variant) {
  std::lock_guard<std::mutex> lk(g_hrr_mu);
  auto key = std::make_tuple(la, lb, lc, bra_pure ? 1 : 0);
  if (variant < 0) g_hrr_hints.erase(key); else g_hrr_hints[key] = variant;
}

int hrr_variant(int la, int lb, int lc, int bra_pure) {
  std::lock_guard<std::mutex> lk(g_hrr_mu);
  auto it = g_hrr_hints.find(std::make_tuple(la, lb, lc, bra_pure ? 1 : 0));
  return it == g_hrr_hints.end() ? 0 : it->second;
}

const ClassTables& class_tables_variant(int la, int lb, int lc, int bra_pure, int hrr2) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, ClassTables> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(la, lb, lc, bra_pure ? 1 : 0, (hrr2 && lb >= 2) ? 1 : 0);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  return cache.emplace(key, build(la, lb, lc, bra_pure ? 1 : 0, std::get<4>(key))).first->second;
}

const ClassTables& class_tables(int la, int lb, int lc, int bra_pure) {
  return class_tables_variant(la, lb, lc, bra_pure, hrr_variant(la, lb, lc, bra_pure));
}

// Invariants of a class's host tables; empty string when they all hold.
std::string check_class_tables(const ClassTables& ct) {
  char buf[160];
  auto bad = [&](const char* what, long long i) {
    std::snprintf(buf, sizeof(buf), "%s (entry %lld)", what, i);
    return std::string(buf);
  };
  const int Lab = ct.la + ct.lb;
  const unsigned NV = (unsigned)ct.NV, NW = (unsigned)ct.NW, NF = (unsigned)ct.NF, NACC = (unsigned)ct.NACC;
  if ((int)ct.vlev_start.size() != Lab + 1) return "VRR1 level table size";
  // VRR1: indices in range; every entry above level 0 written once; level e
  // reads only entries written before it (levels are contiguous and ordered)
  std::vector<int> written(NV, 0);
  for (int e = 1; e <= Lab; ++e) {
    unsigned lo = NV;
    for (int i = ct.vlev_start[e - 1]; i < ct.vlev_start[e]; ++i) lo = std::min(lo, ct.vtab[i].x & 0xFFFF);
    for (int i = ct.vlev_start[e - 1]; i < ct.vlev_start[e]; ++i) {
      const uint4 it = ct.vtab[i];
      const unsigned dst = it.x & 0xFFFF, a = it.x >> 16, an = it.y & 0xFFFF, b = it.y >> 16, bn = it.z & 0xFFFF;
      const unsigned axis = (it.z >> 16) & 0xF, nq = (it.z >> 20) & 0xF;
      if (dst >= NV || a >= lo || an >= lo || axis > 2 || (nq && (b >= lo || bn >= lo)))
        return bad("VRR1 item index out of range or not yet formed", i);
      ++written[dst];
    }
  }
  for (unsigned v = 0; v < NV; ++v)
    if (written[v] != (v <= (unsigned)Lab ? 0 : 1)) return bad("VRR1 entry not formed exactly once", v);
  // weights and accumulators
  for (size_t i = 0; i < ct.wtab.size(); ++i) {
    const int4 w = ct.wtab[i];
    const unsigned cnt = (unsigned)w.z >> 16;
    const unsigned src[4] = {(unsigned)w.x >> 16, (unsigned)w.y & 0xFFFF, (unsigned)w.y >> 16, (unsigned)w.z & 0xFFFF};
    if (((unsigned)w.x & 0xFFFF) >= NW || cnt > 4) return bad("weight item", (long long)i);
    for (unsigned k = 0; k < cnt; ++k)
      if (src[k] >= NF) return bad("weight factor index", (long long)i);
  }
  if (ct.atab.size() != NACC) return "accumulator table size";
  for (size_t i = 0; i < ct.atab.size(); ++i)
    if ((ct.atab[i] & 0xFFFF) >= NV || (ct.atab[i] >> 16) >= NW) return bad("accumulator index", (long long)i);
  // gather: CSR and its sliced-ELL copy hold the same terms
  const int ngt = ct.nkrow * ct.ncc;
  if ((int)ct.gptr.size() != ngt + 1 || (int)ct.gdst.size() != ngt) return "gather table size";
  std::vector<int> seen(ngt, 0);
  for (int r = 0; r < ngt; ++r) {
    if (ct.gdst[r] < 0 || ct.gdst[r] >= ngt || seen[ct.gdst[r]]++) return bad("gather order not a permutation", r);
    if (r && ct.gptr[ct.gdst[r] + 1] - ct.gptr[ct.gdst[r]] > ct.gptr[ct.gdst[r - 1] + 1] - ct.gptr[ct.gdst[r - 1]])
      return bad("gather order not by descending term count", r);
  }
  for (int id = 0; id < ngt; ++id)
    if (ct.gptr[id + 1] < ct.gptr[id]) return bad("gather row pointers", id);
  for (size_t q = 0; q < ct.gterm.size(); ++q)
    if ((ct.gterm[q] & 0xFFFFF) >= NACC || (ct.gterm[q] >> 20) >= ct.pal.size()) return bad("gather term", (long long)q);
  if ((int)ct.gslice.size() != (ngt + 31) / 32) return "sliced ELL slice count";
  for (int sl = 0; sl < (int)ct.gslice.size(); ++sl)
    for (int l = 0; l < 32; ++l) {
      const int r = 32 * sl + l;
      const int id = r < ngt ? ct.gdst[r] : -1;
      const int cnt = id >= 0 ? ct.gptr[id + 1] - ct.gptr[id] : 0;
      if (cnt > ct.gslice[sl].y) return bad("sliced ELL row longer than its slice", r);
      for (int j = 0; j < ct.gslice[sl].y; ++j) {
        const size_t q = (size_t)ct.gslice[sl].x + 32 * j + l;
        if (q >= ct.gell.size()) return bad("sliced ELL entry out of range", r);
        const unsigned e = ct.gell[q];
        if (j < cnt ? e != ct.gterm[ct.gptr[id] + j]
                    : ((e >> 20) >= ct.pal.size() || ct.pal[e >> 20] != 0.0 || (e & 0xFFFFF) >= NACC))
          return bad("sliced ELL differs from the CSR terms", r);
      }
    }
  // ket transform
  if ((int)ct.kptr.size() != ct.nC + 1) return "ket table size";
  for (size_t q = 0; q < ct.kent.size(); ++q)
    if (ct.kent[q].x < 0 || ct.kent[q].x >= ct.ncc || ct.kent[q].y < 0 || ct.kent[q].y >= (int)ct.pal.size())
      return bad("ket entry", (long long)q);
  // HRR: round r rows built from rows of round r-1, 2..4 terms, codes < 13
  for (int r = 1; r <= ct.nhrr; ++r)
    for (int i = ct.hstart[r]; i < ct.hstart[r + 1]; ++i) {
      const uint4 h = ct.htab[i];
      const unsigned nt = h.x >> 16, src[4] = {h.y & 0xFFFF, h.y >> 16, h.z & 0xFFFF, h.z >> 16};
      if ((int)(h.x & 0xFFFF) >= ct.hrows[r] || nt < 2 || nt > 4 || (h.w & 0xF) != 0) return bad("HRR row", i);
      for (unsigned t = 0; t < nt; ++t)
        if ((int)src[t] >= ct.hrows[r - 1] || ((h.w >> (4 * t)) & 0xF) > 12) return bad("HRR term", i);
    }
  if (ct.nhrr != (ct.hrr2 ? ct.lb / 2 + (ct.lb & 1) : ct.lb)) return "HRR round count";
  // bra transforms
  if (ct.nbA)
    for (size_t q = 0; q < ct.baent.size(); ++q)
      if (ct.baent[q].x < 0 || ct.baent[q].x >= ct.ncA) return bad("bra A entry", (long long)q);
  if (ct.nbB)
    for (size_t q = 0; q < ct.bbent.size(); ++q)
      if (ct.bbent[q].x < 0 || ct.bbent[q].x >= ct.ncB) return bad("bra B entry", (long long)q);
  return "";
}

// HRR holds exactly for moment integrals M(a, b) = int (x-A)^a (x-B)^b w(x) dx
// of any weight w, since (x-B) = (x-A) + AB.  With the moments
// mu_k = int (x-A)^k w = 1/(k+1) per axis, feed round 0 the values
// (e 0| = prod_i mu_{e_i}, run the class's HRR rows on the host and compare
// the top round with prod_i sum_j C(b_i, j) AB_i^(b_i-j) mu_{a_i+j}.
double hrr_moment_error(const ClassTables& ct, const double AB[3]) {
  auto mu = [](int k) { return 1.0 / (k + 1); };
  std::vector<double> cur(ct.nkrow);
  for (int r = 0; r < ct.nkrow; ++r)
    cur[r] = mu(ct.erow_xyz[r].x) * mu(ct.erow_xyz[r].y) * mu(ct.erow_xyz[r].z);
  const double c[13] = {1.0, AB[0], AB[1], AB[2], 2 * AB[0], 2 * AB[1], 2 * AB[2], AB[0] * AB[0], AB[1] * AB[1],
                        AB[2] * AB[2], AB[0] * AB[1], AB[0] * AB[2], AB[1] * AB[2]};
  for (int r = 1; r <= ct.nhrr; ++r) {
    std::vector<double> nxt(ct.hrows[r], 0.0);
    for (int i = ct.hstart[r]; i < ct.hstart[r + 1]; ++i) {
      const uint4 h = ct.htab[i];
      const unsigned nt = h.x >> 16, src[4] = {h.y & 0xFFFF, h.y >> 16, h.z & 0xFFFF, h.z >> 16};
      double v = 0;
      for (unsigned t = 0; t < nt; ++t) v += c[(h.w >> (4 * t)) & 0xF] * cur[src[t]];
      nxt[h.x & 0xFFFF] = v;
    }
    cur.swap(nxt);
  }
  double worst = 0;
  auto ca = cart(ct.la), cb = cart(ct.lb);
  for (size_t ia = 0; ia < ca.size(); ++ia)
    for (size_t ib = 0; ib < cb.size(); ++ib) {
      double ref = 1.0, mag = 1.0;
      for (int x = 0; x < 3; ++x) {
        double s = 0, m = 0;
        for (int j = 0; j <= cb[ib].v[x]; ++j) {
          const double t = binom(cb[ib].v[x], j) * std::pow(AB[x], cb[ib].v[x] - j) * mu(ca[ia].v[x] + j);
          s += t;
          m += std::fabs(t);
        }
        ref *= s;
        mag *= m;
      }
      worst = std::max(worst, std::fabs(cur[ia * cb.size() + ib] - ref) / mag);
    }
  return worst;
}

// ---------------------------------------------------------------------------
// Launch shape
// ---------------------------------------------------------------------------

namespace {

struct Sizes {
  long long loop, P, Y, X, pair, aux, total;
};

// per-slot sizes (in doubles) of every stage buffer for a given T, G
void buffer_sizes(const ClassTables& ct, int Kab, int Kc, int T, int G, int mode, Sizes& s,
                  ClassDesc* d) {
  int Tp = (mode == 0 && T > 1) ? (T | 1) : T;
  if (mode == 0 && T > 1 && (T % 2 == 0)) Tp = T + 1;
  auto per_t = [&](int n) -> long long { return mode == 0 ? (long long)n * Tp : (long long)T * n; };
  auto per_tg = [&](int n) -> long long { return mode == 0 ? (long long)n * G * Tp : (long long)T * G * n; };
  long long nK = (long long)ct.nkrow * ct.nC, nG = (long long)ct.nkrow * ct.ncc;
  int lb = ct.lb;
  s.pair = (long long)Kab * kPairRec + 16;  // + the tile's AB products
  s.aux = (long long)T * (3 + kAuxRec * Kc);
  s.loop = per_tg(ct.NV) + per_tg(ct.NW) + per_tg(ct.NF);
  s.P = per_t(ct.NACC);
  // region assignment: Y holds P, level 0 (ket out) and even HRR levels;
  // X holds the loop buffers, the gather output and odd HRR levels.
  long long Y = std::max(s.P, per_t((int)nK));
  long long X = std::max(s.loop, per_t((int)nG));
  const int R = ct.nhrr;
  for (int j = 1; j <= R; ++j) {
    long long sz = per_t(ct.hrows[j] * ct.nC);
    if (j & 1) X = std::max(X, sz); else Y = std::max(Y, sz);
  }
  int cur = (R & 1) ? 1 : 0;  // 0 = Y, 1 = X
  int baR = -1, bbR = -1;
  if (ct.nbA) { cur ^= 1; baR = cur; long long sz = per_t(ct.nbA * ct.nC); if (cur) X = std::max(X, sz); else Y = std::max(Y, sz); }
  if (ct.nbB) { cur ^= 1; bbR = cur; long long sz = per_t(ct.nbB * ct.nC); if (cur) X = std::max(X, sz); else Y = std::max(Y, sz); }
  s.Y = Y;
  s.X = X;
  s.total = s.pair + s.aux + Y + X;
  if (!d) return;
  // fill descriptor layout
  d->T = T; d->Tp = Tp; d->mode = mode; d->G = G;
  d->pair_base = 0;
  d->ab_base = Kab * kPairRec;
  d->aux_base = (int)s.pair;
  int ybase = (int)(s.pair + s.aux);
  int xbase = (int)(ybase + Y);
  auto mk_t = [&](int base, int n) {
    Buf b;
    b.base = base; b.sg = 0;
    if (mode == 0) { b.si = Tp; b.st = 1; } else { b.si = 1; b.st = n; }
    return b;
  };
  auto mk_tg = [&](int base, int n) {
    Buf b;
    b.base = base;
    if (mode == 0) { b.si = G * Tp; b.sg = Tp; b.st = 1; } else { b.si = 1; b.sg = n; b.st = G * n; }
    return b;
  };
  d->V = mk_tg(xbase, ct.NV);
  d->W = mk_tg(xbase + (int)per_tg(ct.NV), ct.NW);
  d->F = mk_tg(xbase + (int)(per_tg(ct.NV) + per_tg(ct.NW)), ct.NF);
  d->P = mk_t(ybase, ct.NACC);
  d->Gb = mk_t(xbase, (int)nG);
  d->H[0] = mk_t(ybase, (int)nK);
  for (int j = 1; j <= R; ++j) d->H[j] = mk_t((j & 1) ? xbase : ybase, ct.hrows[j] * ct.nC);
  Buf last = d->H[R];
  if (ct.nbA) { d->BA = mk_t(baR ? xbase : ybase, ct.nbA * ct.nC); last = d->BA; }
  if (ct.nbB) { d->BB = mk_t(bbR ? xbase : ybase, ct.nbB * ct.nC); last = d->BB; }
  d->OUT = last;
  d->smem_doubles = (int)s.total;
}

}  // namespace

namespace {
std::mutex g_hint_mu;
std::map<std::tuple<int, int, int, int, int, int>, int> g_hints;  // (la, lb, lc, pure, Kab, Kc) -> CTAs/SM
}  // namespace

void set_shape_hint(int la, int lb, int lc, int bra_pure, int Kab, int Kc, int ctas) {
  std::lock_guard<std::mutex> lk(g_hint_mu);
  auto key = std::make_tuple(la, lb, lc, bra_pure ? 1 : 0, Kab, Kc);
  if (ctas <= 0) g_hints.erase(key); else g_hints[key] = ctas;
}

int shape_hint(const ClassTables& ct, int Kab, int Kc) {
  std::lock_guard<std::mutex> lk(g_hint_mu);
  auto it = g_hints.find(std::make_tuple(ct.la, ct.lb, ct.lc, ct.bra_pure ? 1 : 0, Kab, Kc));
  return it == g_hints.end() ? 0 : it->second;
}

namespace {
std::map<std::tuple<int, int, int, int, int, int>, std::pair<int, int>> g_tile_hints;  // -> (T, G)
}  // namespace

void set_tile_hint(int la, int lb, int lc, int bra_pure, int Kab, int Kc, int T, int G) {
  std::lock_guard<std::mutex> lk(g_hint_mu);
  auto key = std::make_tuple(la, lb, lc, bra_pure ? 1 : 0, Kab, Kc);
  if (T <= 0) g_tile_hints.erase(key); else g_tile_hints[key] = {T, G};
}

// The hinted tile (T triples, chunks of G primitives, G balanced over the
// chunks) when one is set for the class and it fits one CTA per SM;
// smem_bytes = -1 otherwise.
LaunchShape tile_hint_shape(const ClassTables& ct, int Kab, int Kc, int smem_limit) {
  std::pair<int, int> h{0, 0};
  {
    std::lock_guard<std::mutex> lk(g_hint_mu);
    auto it = g_tile_hints.find(std::make_tuple(ct.la, ct.lb, ct.lc, ct.bra_pure ? 1 : 0, Kab, Kc));
    if (it != g_tile_hints.end()) h = it->second;
  }
  LaunchShape sh{1, 1, 1, -1};
  if (h.first <= 0) return sh;
  const int K = Kab * Kc, T = h.first;
  int G = std::max(1, std::min(h.second, K));
  const int nch = (K + G - 1) / G;
  G = (K + nch - 1) / nch;
  const int mode = T >= 32 ? 0 : 1;
  Sizes s;
  buffer_sizes(ct, Kab, Kc, T, G, mode, s, nullptr);
  if (s.total * 8 > (long long)smem_limit - 1024) return sh;
  return LaunchShape{T, G, mode, (int)(s.total * 8)};
}

// Largest T (then largest balanced G) whose tile fits `ctas` CTAs per SM,
// falling back to fewer CTAs per SM when nothing fits.
LaunchShape choose_shape_for(const ClassTables& ct, int Kab, int Kc, long long naux, int smem_limit, int ctas) {
  const int K = Kab * Kc;
  std::vector<long long> budgets;
  for (int c = std::max(1, ctas); c >= 1; --c) budgets.push_back((smem_limit / c - 1024) / 8);
  LaunchShape best{1, 1, 1, 0};
  Sizes s;
  int Ts[] = {512, 256, 128, 64, 32, 16, 8, 4, 2, 1};
  bool found = false;
  for (long long budget : budgets) {
    for (int T : Ts) {
      if (T > 1 && T > 2 * naux && T != 1) continue;
      int mode = T >= 32 ? 0 : 1;
      buffer_sizes(ct, Kab, Kc, T, 1, mode, s, nullptr);
      if (s.total > budget) continue;
      // enough independent work per stage?  prefer the largest T that fits
      int G = 1;
      int Gmax = std::min(K, 8);
      while (G < Gmax) {
        buffer_sizes(ct, Kab, Kc, T, G + 1, mode, s, nullptr);
        if (s.total > budget) break;
        ++G;
      }
      // balance the primitive chunks: same number of chunks, equal sizes
      const int nch = (K + G - 1) / G;
      G = (K + nch - 1) / nch;
      buffer_sizes(ct, Kab, Kc, T, G, mode, s, nullptr);
      best = LaunchShape{T, G, mode, (int)(s.total * 8)};
      found = true;
      break;
    }
    if (found) break;
  }
  if (!found) best.smem_bytes = -1;
  return best;
}

// The planner's shape: a tuned tile hint (T, G) for this class, contraction
// and ket contraction when one is set and fits; else two CTAs per SM unless
// a tuned CTAs-per-SM hint says otherwise.
LaunchShape choose_shape(const ClassTables& ct, int Kab, int Kc, long long naux, int smem_limit) {
  const LaunchShape th = tile_hint_shape(ct, Kab, Kc, smem_limit);
  if (th.smem_bytes >= 0) return th;
  const int h = shape_hint(ct, Kab, Kc);
  return choose_shape_for(ct, Kab, Kc, naux, smem_limit, h > 0 ? h : 2);
}

int place_epilogue_scratch(ClassDesc& d, long long need) {
  const bool out_in_x = d.OUT.base == d.V.base;
  const long long free_base = out_in_x ? d.P.base : d.V.base;
  const long long free_size = out_in_x ? (long long)d.V.base - d.P.base : (long long)d.smem_doubles - d.V.base;
  if (need <= free_size) return (int)free_base;
  const int base = d.smem_doubles;
  d.smem_doubles += (int)need;
  return base;
}

void set_digest_scratch(ClassDesc& d) {
  d.dscr = place_epilogue_scratch(d, (long long)d.onA * d.onB + (long long)d.T * d.nC);
}

void fill_layout(ClassDesc& d, const ClassTables& ct, const LaunchShape& sh) {
  Sizes s;
  buffer_sizes(ct, d.Kab, d.Kc, sh.T, sh.G, sh.mode, s, &d);
}

}  // namespace lx3c
