// Host side of the C ABI: context and arena carving, the circuit planner
// (SWAP-chain expansion, single-qubit fusion, gauge moves), the Pauli-term
// trie builder and the entry points declared in tnmps.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <complex>
#include <map>
#include <new>
#include <tuple>

#include "tnmps_internal.h"

using zc = std::complex<double>;

struct tnmps_terms {
  TermPlan plan;
  uint64_t gen = 0;
};

// A super-gate: the gate list with its parameters bound, and the same gates as
// a matrix-product operator over the window [p, q] of qubits they touch.
struct tnmps_supergate {
  int n = 0, p = 0, q = 0;
  std::vector<int> w;             // MPO bonds, w[0] = w[q-p+1] = 1
  std::vector<std::complex<double>> W;  // site tensors [w_{i-1}][2 out][2 in][w_i]
  std::vector<int64_t> woff;      // element offset of each window site
  std::vector<tnmps_gate> gates;  // fixed-angle copy of the gate list
};

namespace {

std::atomic<uint64_t> g_plan_gen{1};
std::atomic<uint64_t> g_ctx_uid{1};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

bool valid_dtype(int d) { return d == TNMPS_C128 || d == TNMPS_C64 || d == TNMPS_C64_BF16SPLIT; }

// bond capacities: cap[i] bounds D_{i-1} (dims index i), cap[0] = cap[n] = 1
std::vector<int> bond_caps(int n, int chi) {
  std::vector<int> cap(n + 1, 1);
  for (int i = 1; i < n; ++i) {
    const int e = std::min(i, n - i);
    cap[i] = e >= 30 ? chi : std::min(chi, 1 << e);
  }
  return cap;
}

struct Layout {
  size_t sites, site_off, dims, theta_buf, w_buf, q_buf, sigma, perm, scale, discarded, theta_dev, err,
      counters, ebuf, tc_a, tc_b, total;
  int64_t tc_a_stride = 0, tc_b_stride = 0;  // per-state bytes of the K2 tensor-core operands
  int64_t state_elems, tw;
  std::vector<int64_t> site_off_h;
  std::vector<int> cap;
};

Layout make_layout(int n, int chi, int dtype, int batch, int max_params) {
  Layout L;
  const size_t esz = dtype == TNMPS_C128 ? 16 : 8;
  L.cap = bond_caps(n, chi);
  L.site_off_h.resize(n);
  int64_t o = 0;
  for (int i = 0; i < n; ++i) {
    L.site_off_h[i] = o;
    o += (int64_t)L.cap[i] * 2 * L.cap[i + 1];
    o = (o + 31) & ~(int64_t)31;
  }
  L.state_elems = o;
  L.tw = (int64_t)(2 * chi) * (2 * chi);
  size_t p = 0;
  L.sites = p;
  p = al256(p + esz * (size_t)batch * (size_t)L.state_elems);
  L.site_off = p;
  p = al256(p + 8 * (size_t)n);
  L.dims = p;
  p = al256(p + 4 * (size_t)batch * (n + 1));
  L.theta_buf = p;
  p = al256(p + esz * (size_t)batch * (size_t)L.tw);
  L.w_buf = p;
  p = al256(p + esz * (size_t)batch * (size_t)L.tw);
  L.q_buf = p;
  p = al256(p + esz * (size_t)batch * (size_t)L.tw);
  L.sigma = p;
  p = al256(p + 8 * (size_t)batch * 2 * chi);
  L.perm = p;
  p = al256(p + 4 * (size_t)batch * 2 * chi);
  L.scale = p;
  p = al256(p + 8 * (size_t)batch);
  L.discarded = p;
  p = al256(p + 8 * (size_t)batch);
  L.theta_dev = p;
  p = al256(p + 8 * (size_t)batch * (size_t)std::max(max_params, 1));
  L.err = p;
  p = al256(p + 4);
  L.counters = p;
  p = al256(p + 8 * CNT_NUM);
  L.ebuf = p;
  if (dtype != TNMPS_C128) p = al256(p + 16 * (size_t)batch * chi * chi);
  L.tc_a = L.tc_b = p;
  if (dtype == TNMPS_C64_BF16SPLIT) {
    L.tc_a_stride = theta_tc_a_bytes(chi);
    L.tc_b_stride = theta_tc_b_bytes(chi);
    p = al256(p + (size_t)batch * (size_t)L.tc_a_stride);
    L.tc_b = p;
    p = al256(p + (size_t)batch * (size_t)L.tc_b_stride);
  }
  L.total = p;
  return L;
}

tnmps_status fail(tnmps_ctx *c, tnmps_status s, const std::string &msg) {
  if (c) c->last_error = msg;
  return s;
}

tnmps_status cuda_fail(tnmps_ctx *c, cudaError_t e, const char *where) {
  return fail(c, TNMPS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

tnmps_status inject(tnmps_ctx *c) {
  ++c->call_count;
  if (c->inject_nth > 0 && c->call_count == c->inject_nth) {
    c->inject_nth = 0;
    return fail(c, c->inject_status, "injected fault");
  }
  return TNMPS_OK;
}

// ------------------------------------------------------------ gate matrices
// Textbook definitions (qubit order of a 4x4: basis 2*s_first + s_second).
void fixed_1q(int op, zc U[4]) {
  const double r = 1.0 / sqrt(2.0);
  const zc I(0, 1);
  switch (op) {
    case TNMPS_I: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = 1; break;
    case TNMPS_X: U[0] = 0; U[1] = 1; U[2] = 1; U[3] = 0; break;
    case TNMPS_Y: U[0] = 0; U[1] = -I; U[2] = I; U[3] = 0; break;
    case TNMPS_Z: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = -1; break;
    case TNMPS_H: U[0] = r; U[1] = r; U[2] = r; U[3] = -r; break;
    case TNMPS_S: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = I; break;
    case TNMPS_SDG: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = -I; break;
    case TNMPS_T: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = std::polar(1.0, M_PI / 4); break;
    default: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = 1;
  }
}

void rot_1q(int op, double a, zc U[4]) {
  const double c = cos(0.5 * a), s = sin(0.5 * a);
  if (op == TNMPS_RX) {
    U[0] = c; U[1] = zc(0, -s); U[2] = zc(0, -s); U[3] = c;
  } else if (op == TNMPS_RY) {
    U[0] = c; U[1] = -s; U[2] = s; U[3] = c;
  } else {
    U[0] = zc(c, -s); U[1] = 0; U[2] = 0; U[3] = zc(c, s);
  }
}

void core_2q(int op, bool first_is_left, zc G[16]) {
  for (int e = 0; e < 16; ++e) G[e] = 0;
  for (int sa = 0; sa < 2; ++sa)
    for (int sb = 0; sb < 2; ++sb) {
      int ta = sa, tb = sb;
      double ph = 1;
      if (op == TNMPS_CNOT) tb = sb ^ sa;
      else if (op == TNMPS_CZ) ph = (sa && sb) ? -1 : 1;
      else { ta = sb; tb = sa; }  // SWAP
      // (sa, sb) are (first, second) operands; map to (left, right) sites
      const int col = first_is_left ? 2 * sa + sb : 2 * sb + sa;
      const int row = first_is_left ? 2 * ta + tb : 2 * tb + ta;
      G[4 * row + col] = ph;
    }
}

bool is_1q(int op) { return op >= TNMPS_I && op <= TNMPS_RZ && op != 11 && op != 12; }
bool is_rot(int op) { return op == TNMPS_RX || op == TNMPS_RY || op == TNMPS_RZ; }
bool is_2q(int op) { return op == TNMPS_CNOT || op == TNMPS_CZ || op == TNMPS_SWAP; }

struct PGate {
  int op, q0, q1, param;
  double angle, scale;
};

Fac1 make_fac(const PGate &g, bool &fixed) {
  Fac1 f;
  memset(&f, 0, sizeof f);
  if (is_rot(g.op) && g.param >= 0) {
    f.kind = g.op == TNMPS_RX ? 1 : g.op == TNMPS_RY ? 2 : 3;
    f.param = g.param;
    f.angle = g.angle;
    f.scale = g.scale;
    fixed = false;
    return f;
  }
  zc U[4];
  if (is_rot(g.op)) rot_1q(g.op, g.angle, U);
  else fixed_1q(g.op, U);
  f.kind = 0;
  f.param = -1;
  for (int e = 0; e < 4; ++e) {
    f.m[2 * e] = U[e].real();
    f.m[2 * e + 1] = U[e].imag();
  }
  fixed = true;
  return f;
}

// append factor to a side list, merging consecutive fixed matrices
void push_fac(std::vector<Fac1> &v, const Fac1 &f) {
  if (f.kind == 0 && !v.empty() && v.back().kind == 0) {
    Fac1 &b = v.back();
    zc A[4], B[4], C[4];
    for (int e = 0; e < 4; ++e) {
      A[e] = zc(f.m[2 * e], f.m[2 * e + 1]);
      B[e] = zc(b.m[2 * e], b.m[2 * e + 1]);
    }
    C[0] = A[0] * B[0] + A[1] * B[2];
    C[1] = A[0] * B[1] + A[1] * B[3];
    C[2] = A[2] * B[0] + A[3] * B[2];
    C[3] = A[2] * B[1] + A[3] * B[3];
    for (int e = 0; e < 4; ++e) {
      b.m[2 * e] = C[e].real();
      b.m[2 * e + 1] = C[e].imag();
    }
    return;
  }
  v.push_back(f);
}

// ------------------------------------------------------- super-gate MPO
// Dense complex matrix, row-major.
struct ZMat {
  int r = 0, c = 0;
  std::vector<zc> a;
  ZMat() = default;
  ZMat(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_) {}
  zc &at(int i, int j) { return a[(size_t)i * c + j]; }
  zc at(int i, int j) const { return a[(size_t)i * c + j]; }
};

// X = Q C with Q (rows x k) orthonormal columns spanning X's columns and
// C = Q^H X: Gram-Schmidt over the columns (two projection passes), a column
// whose remainder is below tol * (largest column norm) adds nothing. k >= 1.
void column_basis(const ZMat &X, double tol, ZMat &Q, ZMat &C) {
  double mx = 0;
  for (int j = 0; j < X.c; ++j) {
    double s = 0;
    for (int i = 0; i < X.r; ++i) s += std::norm(X.at(i, j));
    mx = std::max(mx, sqrt(s));
  }
  std::vector<std::vector<zc>> basis;
  for (int j = 0; j < X.c; ++j) {
    std::vector<zc> v(X.r);
    for (int i = 0; i < X.r; ++i) v[i] = X.at(i, j);
    for (int pass = 0; pass < 2; ++pass)
      for (const auto &b : basis) {
        zc h = 0;
        for (int i = 0; i < X.r; ++i) h += std::conj(b[i]) * v[i];
        for (int i = 0; i < X.r; ++i) v[i] -= h * b[i];
      }
    double nv = 0;
    for (int i = 0; i < X.r; ++i) nv += std::norm(v[i]);
    nv = sqrt(nv);
    if (nv > tol * mx && nv > 0) {
      for (auto &x : v) x /= nv;
      basis.push_back(std::move(v));
    }
  }
  if (basis.empty()) {
    basis.emplace_back(X.r, zc(0));
    basis[0][0] = 1;
  }
  const int k = (int)basis.size();
  Q = ZMat(X.r, k);
  C = ZMat(k, X.c);
  for (int t = 0; t < k; ++t) {
    for (int i = 0; i < X.r; ++i) Q.at(i, t) = basis[t][i];
    for (int j = 0; j < X.c; ++j) {
      zc h = 0;
      for (int i = 0; i < X.r; ++i) h += std::conj(basis[t][i]) * X.at(i, j);
      C.at(t, j) = h;
    }
  }
}

// MPO site tensor T[al][o][s][be]
struct MpoSite {
  int wl = 1, wr = 1;
  std::vector<zc> t;
  zc &at(int al, int o, int s, int be) { return t[(((size_t)al * 2 + o) * 2 + s) * wr + be]; }
};

// Remove linearly dependent directions of every bond: a left-to-right pass
// that reduces each site to an orthonormal column basis of (al o s) x be and
// moves the coefficients into the next site, then the mirror pass from the
// right. The operator is unchanged (up to the tolerance); the bonds become the
// ranks of the operator's cuts.
void compress_mpo(std::vector<MpoSite> &T) {
  const double tol = 1e-13;
  const int m = (int)T.size();
  for (int i = 0; i + 1 < m; ++i) {
    MpoSite &A = T[i], &B = T[i + 1];
    ZMat X(A.wl * 4, A.wr), Q, C;
    for (size_t e = 0; e < A.t.size(); ++e) X.a[e] = A.t[e];
    column_basis(X, tol, Q, C);
    const int k = Q.c;
    A.wr = k;
    A.t = Q.a;
    MpoSite nb;
    nb.wl = k;
    nb.wr = B.wr;
    nb.t.assign((size_t)k * 4 * B.wr, zc(0));
    for (int kk = 0; kk < k; ++kk)
      for (int be = 0; be < B.wl; ++be) {
        const zc f = C.at(kk, be);
        if (f == zc(0)) continue;
        for (size_t r = 0; r < (size_t)4 * B.wr; ++r) nb.t[kk * 4 * B.wr + r] += f * B.t[be * 4 * B.wr + r];
      }
    B = std::move(nb);
  }
  for (int i = m - 1; i > 0; --i) {
    MpoSite &A = T[i], &P = T[i - 1];
    // Z = A^T as (o s be) x al
    ZMat Z(4 * A.wr, A.wl), Q, C;
    for (int al = 0; al < A.wl; ++al)
      for (int r = 0; r < 4 * A.wr; ++r) Z.at(r, al) = A.t[(size_t)al * 4 * A.wr + r];
    column_basis(Z, tol, Q, C);
    const int k = Q.c;
    MpoSite na;
    na.wl = k;
    na.wr = A.wr;
    na.t.assign((size_t)k * 4 * A.wr, zc(0));
    for (int kk = 0; kk < k; ++kk)
      for (int r = 0; r < 4 * A.wr; ++r) na.t[(size_t)kk * 4 * A.wr + r] = Q.at(r, kk);
    A = std::move(na);
    // P[.., al] -> sum_al P[.., al] C[k, al]
    MpoSite np;
    np.wl = P.wl;
    np.wr = k;
    np.t.assign((size_t)P.wl * 4 * k, zc(0));
    for (int row = 0; row < P.wl * 4; ++row)
      for (int kk = 0; kk < k; ++kk) {
        zc acc = 0;
        for (int al = 0; al < P.wr; ++al) acc += P.t[(size_t)row * P.wr + al] * C.at(kk, al);
        np.t[(size_t)row * k + kk] = acc;
      }
    P = std::move(np);
  }
}

// Gate matrix of a (bound) one-qubit gate.
void gate_1q(const tnmps_gate &g, zc U[4]) {
  if (is_rot(g.op)) rot_1q(g.op, g.angle, U);
  else fixed_1q(g.op, U);
}

tnmps_status build_supergate(tnmps_supergate &sg, std::string &err) {
  const int m = sg.q - sg.p + 1;
  std::vector<MpoSite> T(m);
  for (auto &t : T) {
    t.t.assign(4, zc(0));
    t.at(0, 0, 0, 0) = 1;
    t.at(0, 1, 1, 0) = 1;
  }
  for (const tnmps_gate &g : sg.gates) {
    if (is_1q(g.op)) {
      zc U[4];
      gate_1q(g, U);
      MpoSite &A = T[g.q0 - sg.p];
      std::vector<zc> o(A.t.size());
      for (int al = 0; al < A.wl; ++al)
        for (int s = 0; s < 2; ++s)
          for (int be = 0; be < A.wr; ++be)
            for (int oo = 0; oo < 2; ++oo)
              o[(((size_t)al * 2 + oo) * 2 + s) * A.wr + be] =
                  U[2 * oo] * A.at(al, 0, s, be) + U[2 * oo + 1] * A.at(al, 1, s, be);
      A.t = o;
      continue;
    }
    const int qa = std::min(g.q0, g.q1), qb = std::max(g.q0, g.q1);
    zc G[16];
    core_2q(g.op, g.q0 == qa, G);  // basis 2 s_left + s_right
    // M[(oa ia), (ob ib)] = G[(oa ob), (ia ib)] = sum_k A_k[(oa ia)] B_k[(ob ib)]
    ZMat M(4, 4), Q, C;
    for (int oa = 0; oa < 2; ++oa)
      for (int ob = 0; ob < 2; ++ob)
        for (int ia = 0; ia < 2; ++ia)
          for (int ib = 0; ib < 2; ++ib)
            M.at(2 * oa + ia, 2 * ob + ib) = G[4 * (2 * oa + ob) + 2 * ia + ib];
    column_basis(M, 1e-13, Q, C);
    const int r = Q.c;
    const int i = qa - sg.p, j = qb - sg.p;
    for (int site = i; site <= j; ++site) {
      MpoSite &A = T[site];
      MpoSite nA;
      nA.wl = site == i ? A.wl : A.wl * r;
      nA.wr = site == j ? A.wr : A.wr * r;
      nA.t.assign((size_t)nA.wl * 4 * nA.wr, zc(0));
      for (int k = 0; k < r; ++k)
        for (int al = 0; al < A.wl; ++al)
          for (int be = 0; be < A.wr; ++be)
            for (int o = 0; o < 2; ++o)
              for (int s = 0; s < 2; ++s) {
                zc v;
                if (site == i)
                  v = Q.at(2 * o + 0, k) * A.at(al, 0, s, be) + Q.at(2 * o + 1, k) * A.at(al, 1, s, be);
                else if (site == j)
                  v = C.at(k, 2 * o + 0) * A.at(al, 0, s, be) + C.at(k, 2 * o + 1) * A.at(al, 1, s, be);
                else
                  v = A.at(al, o, s, be);
                const int nl = site == i ? al : al * r + k;
                const int nr = site == j ? be : be * r + k;
                nA.at(nl, o, s, nr) = v;
              }
      A = std::move(nA);
    }
    compress_mpo(T);
    for (int site = i; site < j; ++site)
      if (T[site].wr > TNMPS_MAX_MPO_BOND) {
        err = "super-gate MPO bond above " + std::to_string(TNMPS_MAX_MPO_BOND);
        return TNMPS_ERR_UNSUPPORTED;
      }
  }
  sg.w.assign(m + 1, 1);
  sg.woff.assign(m, 0);
  sg.W.clear();
  for (int i = 0; i < m; ++i) {
    sg.woff[i] = (int64_t)sg.W.size();
    sg.w[i + 1] = i + 1 < m ? T[i].wr : 1;
    sg.W.insert(sg.W.end(), T[i].t.begin(), T[i].t.end());
  }
  return TNMPS_OK;
}

}  // namespace

// Plan a gate list for an n-qubit register (see tnmps_internal.h).
tnmps_status plan_gates(int n, const tnmps_gate *gates, size_t n_gates, size_t n_params,
                        std::vector<PlannedOp> &out, std::string &err) {
  auto fail = [&](tnmps_status st, const char *msg) {
    err = msg;
    return st;
  };
  // 1. validate and expand distant two-qubit gates into SWAP chains (Sec. IV)
  std::vector<PGate> ex;
  ex.reserve(n_gates);
  for (size_t k = 0; k < n_gates; ++k) {
    const tnmps_gate &g = gates[k];
    PGate p{g.op, g.q0, g.q1, g.param, g.angle, g.scale};
    if (g.q0 < 0 || g.q0 >= n) return fail(TNMPS_ERR_ARG, "gate qubit out of range");
    if (g.param >= 0 && (size_t)g.param >= n_params)
      return fail(TNMPS_ERR_ARG, "gate parameter index out of range");
    if (is_2q(g.op)) {
      if (g.q1 < 0 || g.q1 >= n || g.q1 == g.q0)
        return fail(TNMPS_ERR_ARG, "bad two-qubit gate operands");
      const int step = g.q1 > g.q0 ? 1 : -1;
      int pos = g.q1;
      std::vector<PGate> chain;
      while (std::abs(pos - g.q0) > 1) {
        chain.push_back(PGate{TNMPS_SWAP, pos, pos - step, -1, 0, 1});
        pos -= step;
      }
      for (auto &s : chain) ex.push_back(s);
      p.q1 = pos;
      ex.push_back(p);
      for (auto it = chain.rbegin(); it != chain.rend(); ++it) ex.push_back(*it);
    } else if (is_1q(g.op)) {
      ex.push_back(p);
    } else {
      return fail(TNMPS_ERR_UNSUPPORTED, "unknown gate opcode");
    }
  }
  // 2. fuse single-qubit runs into the next two-qubit op on the site
  std::vector<std::vector<Fac1>> pend(n);
  auto flush1 = [&](int q) {
    if (pend[q].empty()) return;
    PlannedOp po;
    memset(&po, 0, sizeof po);
    po.two = false;
    po.o1.site = q;
    po.o1.nf = (int)pend[q].size();
    for (int i = 0; i < po.o1.nf; ++i) po.o1.f[i] = pend[q][i];
    out.push_back(po);
    pend[q].clear();
  };
  for (const PGate &g : ex) {
    if (!is_2q(g.op)) {
      bool fixed;
      Fac1 f = make_fac(g, fixed);
      if (g.op == TNMPS_I) continue;
      if ((int)pend[g.q0].size() >= TNMPS_MAX_FAC && !(fixed && pend[g.q0].back().kind == 0))
        flush1(g.q0);
      push_fac(pend[g.q0], f);
      continue;
    }
    const int l = std::min(g.q0, g.q1);
    PlannedOp po;
    memset(&po, 0, sizeof po);
    po.two = true;
    po.o2.l = l;
    zc G[16];
    core_2q(g.op, g.q0 == l, G);
    for (int e = 0; e < 16; ++e) {
      po.o2.core[2 * e] = G[e].real();
      po.o2.core[2 * e + 1] = G[e].imag();
    }
    po.o2.nl = (int)pend[l].size();
    for (int i = 0; i < po.o2.nl; ++i) po.o2.fl[i] = pend[l][i];
    po.o2.nr = (int)pend[l + 1].size();
    for (int i = 0; i < po.o2.nr; ++i) po.o2.fr[i] = pend[l + 1][i];
    pend[l].clear();
    pend[l + 1].clear();
    out.push_back(po);
  }
  for (int q = 0; q < n; ++q) flush1(q);
  return TNMPS_OK;
}

namespace {

tnmps_status sync_check(tnmps_ctx *c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  uint32_t flags = 0;
  e = cudaMemcpy(&flags, c->err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "read error flags");
  if (flags & TNMPS_EFLAG_NUMERIC)
    return fail(c, TNMPS_ERR_NUMERIC, "NaN/Inf in singular values or energies");
  if (flags & TNMPS_EFLAG_NOT_CONVERGED)
    return fail(c, TNMPS_ERR_NOT_CONVERGED, "Jacobi SVD reached its sweep cap");
  if (flags & TNMPS_EFLAG_TIMEOUT)
    return fail(c, TNMPS_ERR_TIMEOUT,
                "a device-side wait ran out (tensor-core pipeline stalled); results invalid");
  return TNMPS_OK;
}

tnmps_status move_centre(tnmps_ctx *c, int target) {
  if (c->centre < 0) {  // product state: every site is already an isometry
    c->centre = target;
    return TNMPS_OK;
  }
  while (c->centre < target) {
    cudaError_t e = launch_move_right(c, c->centre);
    if (e != cudaSuccess) return cuda_fail(c, e, "QR move");
    ++c->centre;
  }
  while (c->centre > target) {
    cudaError_t e = launch_move_left(c, c->centre);
    if (e != cudaSuccess) return cuda_fail(c, e, "LQ move");
    --c->centre;
  }
  return TNMPS_OK;
}

tnmps_status run_circuit(tnmps_ctx *c, const tnmps_gate *gates, size_t n_gates,
                         const double *theta_dev, int64_t ths, size_t n_params) {
  std::vector<PlannedOp> ops;
  tnmps_status st = plan_gates(c->n, gates, n_gates, n_params, ops, c->last_error);
  if (st != TNMPS_OK) return st;
  for (const PlannedOp &po : ops) {
    if (po.two) {
      if ((st = move_centre(c, po.o2.l)) != TNMPS_OK) return st;
      cudaError_t e = launch_gate2(c, po.o2, theta_dev, ths);
      if (e != cudaSuccess) return cuda_fail(c, e, "two-qubit gate");
      c->centre = po.o2.l + 1;
    } else {
      cudaError_t e = launch_gate1(c, po.o1, theta_dev, ths);
      if (e != cudaSuccess) return cuda_fail(c, e, "one-qubit gate");
    }
  }
  return TNMPS_OK;
}

tnmps_status reset_state(tnmps_ctx *c) {
  cudaError_t e = cudaMemsetAsync(c->err, 0, 4, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->counters, 0, 8 * CNT_NUM, c->stream);
  if (e == cudaSuccess) e = launch_init_state(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "reset");
  c->centre = -1;
  c->ub.assign(c->n + 1, 1);
  return TNMPS_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

const char *tnmps_status_string(tnmps_status s) {
  switch (s) {
    case TNMPS_OK: return "ok";
    case TNMPS_ERR_ARG: return "invalid argument";
    case TNMPS_ERR_NOMEM: return "arena or workspace too small";
    case TNMPS_ERR_UNSUPPORTED: return "unsupported";
    case TNMPS_ERR_NOT_CONVERGED: return "SVD did not converge";
    case TNMPS_ERR_NUMERIC: return "non-finite values";
    case TNMPS_ERR_CUDA: return "CUDA error";
    case TNMPS_ERR_INJECTED: return "injected fault";
    case TNMPS_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char *tnmps_version(void) { return "tnmps 0.1 (sm_103a)"; }

size_t tnmps_state_bytes(int n, int chi, tnmps_dtype dtype, int batch, int max_params) {
  if (n < 1 || n > 4096 || chi < 1 || chi > TNMPS_MAX_CHI || batch < 1 || max_params < 0 ||
      !valid_dtype(dtype))
    return 0;
  return make_layout(n, chi, dtype, batch, max_params).total;
}

tnmps_status tnmps_init(tnmps_ctx **out, int n, int chi, tnmps_dtype dtype, int batch,
                        int max_params, void *arena, size_t arena_bytes) {
  if (!out) return TNMPS_ERR_ARG;
  *out = nullptr;
  const size_t need = tnmps_state_bytes(n, chi, dtype, batch, max_params);
  if (need == 0) return TNMPS_ERR_ARG;
  if (!arena || ((uintptr_t)arena & 255)) return TNMPS_ERR_ARG;
  if (arena_bytes < need) return TNMPS_ERR_NOMEM;
  tnmps_ctx *c = new (std::nothrow) tnmps_ctx();
  if (!c) return TNMPS_ERR_NOMEM;
  Layout L = make_layout(n, chi, dtype, batch, max_params);
  c->uid = g_ctx_uid++;
  c->n = n;
  c->chi = chi;
  c->batch = batch;
  c->max_params = max_params;
  c->dtype = dtype;
  c->arena = (char *)arena;
  c->arena_bytes = arena_bytes;
  c->sites = c->arena + L.sites;
  c->site_off_dev = (int64_t *)(c->arena + L.site_off);
  c->dims = (int32_t *)(c->arena + L.dims);
  c->theta_buf = c->arena + L.theta_buf;
  c->w_buf = c->arena + L.w_buf;
  c->q_buf = c->arena + L.q_buf;
  c->sigma = (double *)(c->arena + L.sigma);
  c->perm = (int32_t *)(c->arena + L.perm);
  c->scale = (double *)(c->arena + L.scale);
  c->discarded = (double *)(c->arena + L.discarded);
  c->theta_dev = (double *)(c->arena + L.theta_dev);
  c->err = (uint32_t *)(c->arena + L.err);
  c->counters = (unsigned long long *)(c->arena + L.counters);
  c->ebuf = c->arena + L.ebuf;
  c->tc_a = c->arena + L.tc_a;
  c->tc_b = c->arena + L.tc_b;
  c->tc_a_stride = L.tc_a_stride;
  c->tc_b_stride = L.tc_b_stride;
  c->site_off = L.site_off_h;
  c->cap = L.cap;
  c->state_elems = L.state_elems;
  c->tw = L.tw;
  cudaError_t e = cudaMemcpy(c->site_off_dev, c->site_off.data(), 8 * (size_t)n,
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete c;
    return TNMPS_ERR_CUDA;
  }
  tnmps_status st = reset_state(c);
  if (st == TNMPS_OK) st = sync_check(c);
  if (st != TNMPS_OK) {
    delete c;
    return st;
  }
  *out = c;
  return TNMPS_OK;
}

void tnmps_free(tnmps_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto &r : c->prof_open) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

tnmps_status tnmps_set_cutoff(tnmps_ctx *c, double eps) {
  if (!c || !(eps >= 0) || !isfinite(eps)) return fail(c, TNMPS_ERR_ARG, "bad cutoff");
  c->eps = eps;
  return TNMPS_OK;
}

tnmps_status tnmps_set_stream(tnmps_ctx *c, void *stream) {
  if (!c) return TNMPS_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  return TNMPS_OK;
}

tnmps_status tnmps_reset(tnmps_ctx *c) {
  if (!c) return TNMPS_ERR_ARG;
  tnmps_status st = inject(c);
  if (st != TNMPS_OK) return st;
  return reset_state(c);
}

static tnmps_status apply_common(tnmps_ctx *c, const tnmps_gate *gates, size_t n_gates,
                                 const double *th, size_t n_params, int mode) {
  // mode 0: host theta shared; 1: host theta per state; 2: device theta per state
  if (!c || (n_gates && !gates)) return fail(c, TNMPS_ERR_ARG, "null argument");
  tnmps_status st = inject(c);
  if (st != TNMPS_OK) return st;
  if (n_params > 0 && !th) return fail(c, TNMPS_ERR_ARG, "null theta");
  if (mode != 2 && n_params > (size_t)c->max_params)
    return fail(c, TNMPS_ERR_ARG, "n_params exceeds the context's max_params");
  const double *thd = nullptr;
  int64_t ths = 0;
  if (n_params > 0) {
    if (mode == 2) {
      thd = th;
      ths = (int64_t)n_params;
    } else {
      const size_t rows = mode == 0 ? 1 : (size_t)c->batch;
      cudaError_t e = cudaMemcpyAsync(c->theta_dev, th, 8 * rows * n_params,
                                      cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "theta upload");
      thd = c->theta_dev;
      ths = mode == 0 ? 0 : (int64_t)n_params;
    }
  }
  st = run_circuit(c, gates, n_gates, thd, ths, n_params);
  if (st != TNMPS_OK) return st;
  return mode == 2 ? TNMPS_OK : sync_check(c);
}

tnmps_status tnmps_apply_circuit(tnmps_ctx *c, const tnmps_gate *g, size_t ng, const double *th,
                                 size_t np) {
  return apply_common(c, g, ng, th, np, 0);
}
tnmps_status tnmps_apply_circuit_batched(tnmps_ctx *c, const tnmps_gate *g, size_t ng,
                                         const double *th, size_t np) {
  return apply_common(c, g, ng, th, np, 1);
}
tnmps_status tnmps_apply_circuit_batched_dev(tnmps_ctx *c, const tnmps_gate *g, size_t ng,
                                             const double *th, size_t np) {
  return apply_common(c, g, ng, th, np, 2);
}

tnmps_status tnmps_terms_create(tnmps_terms **out, int n, const int32_t *off, const int32_t *sites,
                                const uint8_t *paulis, const double *coeffs, size_t T) {
  if (!out || n < 1 || !off || (T && !coeffs)) return TNMPS_ERR_ARG;
  *out = nullptr;
  if (off[0] != 0) return TNMPS_ERR_ARG;
  for (size_t k = 0; k < T; ++k)
    if (off[k + 1] < off[k]) return TNMPS_ERR_ARG;
  if (off[T] > 0 && (!sites || !paulis)) return TNMPS_ERR_ARG;
  tnmps_terms *tt = new (std::nothrow) tnmps_terms();
  if (!tt) return TNMPS_ERR_NOMEM;
  TermPlan &p = tt->plan;
  p.n = n;
  p.n_terms = (int64_t)T;
  p.coeffs.assign(coeffs, coeffs + T);
  // global trie: key (parent global id or -1-start, pauli) -> global id
  struct Node {
    int32_t site, level;
    int64_t parent;
    uint8_t pauli;
  };
  std::vector<Node> nodes;
  std::map<std::pair<int64_t, int>, int64_t> child;
  std::vector<std::pair<int64_t, int>> attach;  // (term, global node)
  std::vector<int32_t> ops(n);
  for (size_t k = 0; k < T; ++k) {
    const int32_t a0 = off[k], a1 = off[k + 1];
    if (a0 == a1) {
      p.identity_terms.push_back((int32_t)k);
      continue;
    }
    std::fill(ops.begin(), ops.end(), 0);
    int lo = n, hi = -1;
    for (int32_t j = a0; j < a1; ++j) {
      const int s = sites[j], q = paulis[j];
      if (s < 0 || s >= n || q < 1 || q > 3 || ops[s] != 0) {
        delete tt;
        return TNMPS_ERR_ARG;
      }
      ops[s] = q;
      lo = std::min(lo, s);
      hi = std::max(hi, s);
    }
    int64_t cur = -1 - (int64_t)lo;
    for (int s = lo; s <= hi; ++s) {
      auto key = std::make_pair(cur, ops[s]);
      auto it = child.find(key);
      if (it == child.end()) {
        Node nd{s, s - lo + 1, cur >= 0 ? cur : -1, (uint8_t)ops[s]};
        nodes.push_back(nd);
        it = child.emplace(key, (int64_t)nodes.size() - 1).first;
      }
      cur = it->second;
    }
    attach.emplace_back((int64_t)k, cur);
  }
  int32_t depth = 0;
  for (auto &nd : nodes) depth = std::max(depth, nd.level);
  p.depth = depth;
  // level-local numbering in creation order
  std::vector<int64_t> local(nodes.size());
  std::vector<int64_t> count(depth + 1, 0);
  for (size_t g = 0; g < nodes.size(); ++g) local[g] = count[nodes[g].level]++;
  p.level_start.assign(depth + 1, 0);
  for (int d = 1; d <= depth; ++d) p.level_start[d] = p.level_start[d - 1] + count[d];
  p.node_site.assign(nodes.size(), 0);
  p.node_parent.assign(nodes.size(), -1);
  p.node_pauli.assign(nodes.size(), 0);
  for (size_t g = 0; g < nodes.size(); ++g) {
    const int64_t pos = p.level_start[nodes[g].level - 1] + local[g];
    p.node_site[pos] = nodes[g].site;
    p.node_parent[pos] = nodes[g].parent >= 0 ? (int32_t)local[nodes[g].parent] : -1;
    p.node_pauli[pos] = nodes[g].pauli;
  }
  for (int d = 1; d <= depth; ++d) p.max_level_nodes = std::max(p.max_level_nodes, count[d]);
  // terms grouped by the level of their node
  std::vector<std::vector<std::pair<int64_t, int64_t>>> bylevel(depth + 1);
  for (auto &at : attach) bylevel[nodes[at.second].level].push_back(at);
  p.tlevel_start.assign(depth + 1, 0);
  for (int d = 1; d <= depth; ++d) {
    for (auto &at : bylevel[d]) {
      p.tterm.push_back((int32_t)at.first);
      p.tnode.push_back((int32_t)local[at.second]);
      p.tsite.push_back(nodes[at.second].site);
    }
    p.tlevel_start[d] = (int64_t)p.tterm.size();
    p.max_level_terms = std::max(p.max_level_terms, (int64_t)bylevel[d].size());
  }
  tt->gen = g_plan_gen++;
  *out = tt;
  return TNMPS_OK;
}

void tnmps_terms_free(tnmps_terms *t) { delete t; }

tnmps_status tnmps_terms_info(const tnmps_terms *t, int64_t *n_nodes, int32_t *depth,
                              int64_t *max_level_nodes) {
  if (!t) return TNMPS_ERR_ARG;
  if (n_nodes) *n_nodes = (int64_t)t->plan.node_site.size();
  if (depth) *depth = t->plan.depth;
  if (max_level_nodes) *max_level_nodes = t->plan.max_level_nodes;
  return TNMPS_OK;
}

size_t tnmps_expect_workspace_bytes(const tnmps_ctx *c, const tnmps_terms *t, int chunk) {
  if (!c || !t || t->plan.n != c->n || chunk < 0) return 0;
  return expect_ws_bytes(c, t->plan, chunk);
}

static tnmps_status expect_common(tnmps_ctx *c, const tnmps_terms *t, void *ws, size_t wsb,
                                  double *energy_dev, double *per_term_dev,
                                  double **energy_used = nullptr,
                                  double **per_term_used = nullptr) {
  if (!c || !t || !ws) return fail(c, TNMPS_ERR_ARG, "null argument");
  if (t->plan.n != c->n) return fail(c, TNMPS_ERR_ARG, "term set built for another register");
  if ((uintptr_t)ws & 255) return fail(c, TNMPS_ERR_ARG, "workspace not 256-byte aligned");
  tnmps_status st = inject(c);
  if (st != TNMPS_OK) return st;
  if ((st = move_centre(c, c->n - 1)) != TNMPS_OK) return st;
  if (c->plan_gen != t->gen) c->plan_terms = nullptr;
  c->plan_gen = t->gen;
  cudaError_t e = expect_run(c, t->plan, (char *)ws, wsb, 0, energy_dev, per_term_dev,
                             energy_used, per_term_used);
  if (e == cudaErrorMemoryAllocation) return fail(c, TNMPS_ERR_NOMEM, "workspace too small");
  if (e != cudaSuccess) return cuda_fail(c, e, "expectation");
  return TNMPS_OK;
}

tnmps_status tnmps_expect_pauli_sum_dev(tnmps_ctx *c, const tnmps_terms *t, void *ws, size_t wsb,
                                        double *energy_dev, double *per_term_dev) {
  if (!energy_dev) return fail(c, TNMPS_ERR_ARG, "null energy");
  return expect_common(c, t, ws, wsb, energy_dev, per_term_dev);
}

tnmps_status tnmps_expect_pauli_sum(tnmps_ctx *c, const tnmps_terms *t, void *ws, size_t wsb,
                                    double *energy, double *per_term) {
  if (!c || !t || !energy) return fail(c, TNMPS_ERR_ARG, "null argument");
  // results land in the workspace's own per-term/energy regions, then to host
  const size_t need_min = tnmps_expect_workspace_bytes(c, t, 1);
  if (wsb < need_min) return fail(c, TNMPS_ERR_NOMEM, "workspace too small");
  double *en = nullptr, *pt = nullptr;
  tnmps_status st = expect_common(c, t, ws, wsb, nullptr, nullptr, &en, &pt);
  if (st != TNMPS_OK) return st;
  cudaError_t e = cudaMemcpyAsync(energy, en, 8 * (size_t)c->batch, cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess && per_term)
    e = cudaMemcpyAsync(per_term, pt, 8 * (size_t)c->batch * t->plan.n_terms,
                        cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "result download");
  return sync_check(c);
}

tnmps_status tnmps_expect_pauli_sum_noalloc(tnmps_ctx *c, const tnmps_terms *t,
                                            double *energy_dev, double *per_term_dev) {
  if (!c || !t || !energy_dev) return fail(c, TNMPS_ERR_ARG, "null argument");
  if (t->plan.n != c->n) return fail(c, TNMPS_ERR_ARG, "term set built for another register");
  tnmps_status st = inject(c);
  if (st != TNMPS_OK) return st;
  if ((st = move_centre(c, c->n - 1)) != TNMPS_OK) return st;
  return expect_noalloc_impl(c, t->plan, t->gen, energy_dev, per_term_dev);
}

tnmps_status tnmps_sample_dev(tnmps_ctx *c, const double *uniforms_dev, int shots,
                              uint8_t *bits_dev) {
  if (!c) return TNMPS_ERR_ARG;
  if (!uniforms_dev || !bits_dev) return fail(c, TNMPS_ERR_ARG, "null pointer");
  if (shots < 1) return fail(c, TNMPS_ERR_ARG, "shots < 1");
  tnmps_status st = inject(c);
  if (st != TNMPS_OK) return st;
  if ((st = move_centre(c, c->n - 1)) != TNMPS_OK) return st;
  cudaError_t e = launch_sample(c, uniforms_dev, shots, bits_dev);
  return e == cudaSuccess ? TNMPS_OK : cuda_fail(c, e, "sample");
}

// ---------------------------------------------------------- super-gates
tnmps_status tnmps_supergate_create(tnmps_supergate **out, int n, const tnmps_gate *gates,
                                    size_t n_gates, const double *theta, size_t n_params) {
  if (!out) return TNMPS_ERR_ARG;
  *out = nullptr;
  if (n < 1 || n_gates == 0 || !gates || (n_params && !theta)) return TNMPS_ERR_ARG;
  tnmps_supergate *sg = new (std::nothrow) tnmps_supergate();
  if (!sg) return TNMPS_ERR_NOMEM;
  sg->n = n;
  sg->p = n;
  sg->q = -1;
  for (size_t k = 0; k < n_gates; ++k) {
    tnmps_gate g = gates[k];
    const bool two = is_2q(g.op);
    if ((!two && !is_1q(g.op)) || g.q0 < 0 || g.q0 >= n ||
        (two && (g.q1 < 0 || g.q1 >= n || g.q1 == g.q0)) ||
        (g.param >= 0 && (size_t)g.param >= n_params)) {
      delete sg;
      return TNMPS_ERR_ARG;
    }
    if (g.param >= 0) {  // bind the parameter: a fixed-angle rotation
      g.angle += g.scale * theta[g.param];
      g.param = -1;
      g.scale = 1;
    }
    if (!two) g.q1 = -1;
    sg->p = std::min(sg->p, two ? std::min(g.q0, g.q1) : g.q0);
    sg->q = std::max(sg->q, two ? std::max(g.q0, g.q1) : g.q0);
    sg->gates.push_back(g);
  }
  std::string err;
  tnmps_status st = build_supergate(*sg, err);
  if (st != TNMPS_OK) {
    delete sg;
    return st;
  }
  *out = sg;
  return TNMPS_OK;
}

void tnmps_supergate_free(tnmps_supergate *sg) { delete sg; }

tnmps_status tnmps_supergate_info(const tnmps_supergate *sg, int32_t *first, int32_t *last,
                                  int32_t *bonds) {
  if (!sg) return TNMPS_ERR_ARG;
  if (first) *first = sg->p;
  if (last) *last = sg->q;
  if (bonds)
    for (size_t i = 0; i < sg->w.size(); ++i) bonds[i] = sg->w[i];
  return TNMPS_OK;
}

tnmps_status tnmps_supergate_mpo(const tnmps_supergate *sg, double *out, size_t cap) {
  if (!sg || !out) return TNMPS_ERR_ARG;
  if (cap < 2 * sg->W.size()) return TNMPS_ERR_NOMEM;
  for (size_t e = 0; e < sg->W.size(); ++e) {
    out[2 * e] = sg->W[e].real();
    out[2 * e + 1] = sg->W[e].imag();
  }
  return TNMPS_OK;
}

namespace {

// Workspace of a fit: psi snapshot, psi dims, MPO, environments, three
// scratch buffers, overlaps and the saved discarded weights.
struct FitLayout {
  size_t psi, pdims, mpo, env, s1, s2, s3, ov, saved, total;
  int64_t psi_stride, env_stride, s_stride;
  std::vector<int64_t> env_off;
};

FitLayout fit_layout(const tnmps_ctx *c, const tnmps_supergate *sg) {
  FitLayout L;
  const size_t esz = c->dtype == TNMPS_C128 ? 16 : 8;
  const int p = sg->p, q = sg->q, B = c->batch;
  const int64_t end = q + 1 < c->n ? c->site_off[q + 1] : c->state_elems;
  L.psi_stride = end - c->site_off[p];
  auto cap = [&](int dims_index) { return (int64_t)c->cap[dims_index]; };
  auto w = [&](int bond) { return (int64_t)sg->w[bond + 1 - p]; };  // bonds p-1..q
  L.env_stride = 0;
  for (int b = p - 1; b <= q; ++b) {
    L.env_off.push_back(L.env_stride);
    L.env_stride += cap(b + 1) * w(b) * cap(b + 1);
    L.env_stride = (L.env_stride + 31) & ~(int64_t)31;
  }
  int64_t s = 0;
  for (int i = p; i <= q; ++i) {
    const int64_t Ca = cap(i), Cm = cap(i + 1), wa = w(i - 1), wm = w(i);
    s = std::max(s, Ca * wa * 2 * Cm);   // T1
    s = std::max(s, Ca * 2 * wm * Cm);   // T2
    s = std::max(s, 2 * Ca * Cm * wm);   // V1
    s = std::max(s, 2 * Cm * wa * Ca);   // V2
    if (i < q) {
      const int64_t Cc = cap(i + 2), wc = w(i + 1);
      s = std::max(s, Ca * 2 * wm * 2 * Cc);  // T3
      s = std::max(s, 4 * Ca * wc * Cc);      // T4
    }
  }
  L.s_stride = (s + 31) & ~(int64_t)31;
  size_t o = 0;
  L.psi = o;
  o = al256(o + esz * B * L.psi_stride);
  L.pdims = o;
  o = al256(o + 4 * (size_t)B * (c->n + 1));
  L.mpo = o;
  o = al256(o + esz * sg->W.size());
  L.env = o;
  o = al256(o + esz * B * L.env_stride);
  L.s1 = o;
  o = al256(o + esz * B * L.s_stride);
  L.s2 = o;
  o = al256(o + esz * B * L.s_stride);
  L.s3 = o;
  o = al256(o + esz * B * L.s_stride);
  L.ov = o;
  o = al256(o + 16 * (size_t)B);
  L.saved = o;
  o = al256(o + 8 * (size_t)B);
  L.total = o;
  return L;
}

}  // namespace

size_t tnmps_supergate_workspace_bytes(const tnmps_ctx *c, const tnmps_supergate *sg) {
  if (!c || !sg || sg->n != c->n) return 0;
  return fit_layout(c, sg).total;
}

tnmps_status tnmps_apply_supergate(tnmps_ctx *c, const tnmps_supergate *sg, int chi_max,
                                   double target, double tol, int max_sweeps, void *ws,
                                   size_t ws_bytes, double *fidelity, double *fidelity_start,
                                   int32_t *info) {
  if (!c) return TNMPS_ERR_ARG;
  if (!sg || sg->n != c->n) return fail(c, TNMPS_ERR_ARG, "super-gate for another register");
  if (chi_max < 1 || chi_max > c->chi) return fail(c, TNMPS_ERR_ARG, "chi_max outside 1..chi");
  if (max_sweeps < 1) return fail(c, TNMPS_ERR_ARG, "max_sweeps < 1");
  tnmps_status st = inject(c);
  if (st != TNMPS_OK) return st;
  const int B = c->batch, p = sg->p, q = sg->q;
  std::vector<double> F(B, 1.0), F0(B, 1.0), Fprev(B, 0.0), ovh(2 * (size_t)B);
  int sweeps = 0, stages = 0, chi = 0;
  auto outputs = [&]() {
    if (fidelity) std::copy(F.begin(), F.end(), fidelity);
    if (fidelity_start) std::copy(F0.begin(), F0.end(), fidelity_start);
    if (info) {
      info[0] = sweeps;
      info[1] = stages;
      info[2] = chi;
    }
  };
  if (p == q) {  // one qubit: the gates apply exactly
    if ((st = run_circuit(c, sg->gates.data(), sg->gates.size(), nullptr, 0, 0)) != TNMPS_OK)
      return st;
    if ((st = sync_check(c)) != TNMPS_OK) return st;
    outputs();
    return TNMPS_OK;
  }
  const FitLayout L = fit_layout(c, sg);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(c, TNMPS_ERR_ARG, "workspace null or not 256-byte aligned");
  if (ws_bytes < L.total) return fail(c, TNMPS_ERR_NOMEM, "super-gate workspace too small");
  if ((st = move_centre(c, p)) != TNMPS_OK) return st;
  char *w8 = static_cast<char *>(ws);
  const size_t esz = c->dtype == TNMPS_C128 ? 16 : 8;
  FitDev f;
  f.p = p;
  f.q = q;
  f.psi = w8 + L.psi;
  f.psi_stride = L.psi_stride;
  f.psi_base = c->site_off[p];
  f.pdims = reinterpret_cast<const int32_t *>(w8 + L.pdims);
  f.s1 = w8 + L.s1;
  f.s2 = w8 + L.s2;
  f.s3 = w8 + L.s3;
  f.s_stride = L.s_stride;
  f.env = w8 + L.env;
  f.env_stride = L.env_stride;
  f.mpo = w8 + L.mpo;
  f.mpo_off = sg->woff;
  f.w = sg->w;
  f.env_off = L.env_off;
  f.pub = c->ub;
  double *ov = reinterpret_cast<double *>(w8 + L.ov);
  double *saved = reinterpret_cast<double *>(w8 + L.saved);
  // MPO in the context's precision (host copy kept alive until the first sync)
  std::vector<double> mpo_d;
  std::vector<float> mpo_f;
  const void *mpo_src;
  if (c->dtype == TNMPS_C128) {
    mpo_d.resize(2 * sg->W.size());
    for (size_t e = 0; e < sg->W.size(); ++e) {
      mpo_d[2 * e] = sg->W[e].real();
      mpo_d[2 * e + 1] = sg->W[e].imag();
    }
    mpo_src = mpo_d.data();
  } else {
    mpo_f.resize(2 * sg->W.size());
    for (size_t e = 0; e < sg->W.size(); ++e) {
      mpo_f[2 * e] = (float)sg->W[e].real();
      mpo_f[2 * e + 1] = (float)sg->W[e].imag();
    }
    mpo_src = mpo_f.data();
  }
  char *sites = static_cast<char *>(c->sites);
  const size_t row = esz * (size_t)L.psi_stride, pitch = esz * (size_t)c->state_elems;
  cudaError_t e = cudaMemcpyAsync(w8 + L.mpo, mpo_src, esz * sg->W.size(),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(w8 + L.psi, row, sites + esz * c->site_off[p], pitch, row, B,
                          cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w8 + L.pdims, c->dims, 4 * (size_t)B * (c->n + 1),
                        cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(saved, c->discarded, 8 * (size_t)B, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "super-gate snapshot");
  const std::vector<int> ub0 = c->ub;
  // step (6) starts from the bonds of the copy of step (3)
  chi = 1;
  for (int b = p; b < q; ++b) chi = std::max(chi, c->ub[b + 1]);
  chi = std::min(chi, chi_max);
  auto read_fidelity = [&](std::vector<double> &out) -> tnmps_status {
    cudaError_t e2 = cudaMemcpyAsync(ovh.data(), ov, 16 * (size_t)B, cudaMemcpyDeviceToHost,
                                     c->stream);
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "read overlaps");
    tnmps_status s2 = sync_check(c);
    if (s2 != TNMPS_OK) return s2;
    for (int b = 0; b < B; ++b) out[b] = ovh[2 * b] * ovh[2 * b] + ovh[2 * b + 1] * ovh[2 * b + 1];
    return TNMPS_OK;
  };
  for (;;) {
    ++stages;
    if (stages > 1) {  // back to the copy of psi
      e = cudaMemcpy2DAsync(sites + esz * c->site_off[p], pitch, w8 + L.psi, row, row, B,
                            cudaMemcpyDeviceToDevice, c->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->dims, w8 + L.pdims, 4 * (size_t)B * (c->n + 1),
                            cudaMemcpyDeviceToDevice, c->stream);
      if (e != cudaSuccess) {
        c->fit_cap = 0;
        return cuda_fail(c, e, "super-gate restore");
      }
      c->ub = ub0;
      c->centre = p;
    }
    // first iterate: the gates one by one under the stage's bond cap
    c->fit_cap = chi;
    st = run_circuit(c, sg->gates.data(), sg->gates.size(), nullptr, 0, 0);
    if (st == TNMPS_OK && (e = fit_overlap(c, f, ov)) != cudaSuccess)
      st = cuda_fail(c, e, "super-gate overlap");
    if (st == TNMPS_OK) st = read_fidelity(F0);
    if (st != TNMPS_OK) {
      c->fit_cap = 0;
      return st;
    }
    F = F0;
    for (int sw = 0; sw < max_sweeps; ++sw) {
      if ((st = move_centre(c, p)) == TNMPS_OK) {
        if ((e = fit_sweep(c, f, ov)) != cudaSuccess) st = cuda_fail(c, e, "super-gate sweep");
        c->centre = q;
      }
      if (st == TNMPS_OK) st = read_fidelity(F);
      if (st != TNMPS_OK) {
        c->fit_cap = 0;
        return st;
      }
      ++sweeps;
      double gain = -1e300;
      for (int b = 0; b < B; ++b) gain = std::max(gain, F[b] - Fprev[b]);
      if (sw > 0 && gain < tol) break;
      Fprev = F;
    }
    double worst = 0;
    for (int b = 0; b < B; ++b) worst = std::max(worst, 1.0 - F[b]);
    if (worst <= target || chi >= chi_max) break;
    chi = std::min(chi_max, 2 * chi);
  }
  c->fit_cap = 0;
  if ((e = fit_finish(c, saved, ov)) != cudaSuccess) return cuda_fail(c, e, "super-gate finish");
  if ((st = sync_check(c)) != TNMPS_OK) return st;
  outputs();
  return TNMPS_OK;
}

tnmps_status tnmps_check(tnmps_ctx *c) {
  if (!c) return TNMPS_ERR_ARG;
  return sync_check(c);
}

tnmps_status tnmps_get_bond_dims(tnmps_ctx *c, int32_t *dims) {
  if (!c || !dims) return TNMPS_ERR_ARG;
  std::vector<int32_t> all((size_t)c->batch * (c->n + 1));
  cudaError_t e = cudaMemcpyAsync(all.data(), c->dims, 4 * all.size(), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "read dims");
  for (int b = 0; b < c->batch; ++b)
    for (int i = 0; i < c->n - 1; ++i) dims[(size_t)b * (c->n - 1) + i] = all[(size_t)b * (c->n + 1) + i + 1];
  return TNMPS_OK;
}

tnmps_status tnmps_get_discarded_weight(tnmps_ctx *c, double *w) {
  if (!c || !w) return TNMPS_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(w, c->discarded, 8 * (size_t)c->batch, cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "read discarded weight");
  return TNMPS_OK;
}

tnmps_status tnmps_get_site(tnmps_ctx *c, int b, int site, double *out, size_t cap, int32_t *dl,
                            int32_t *dr) {
  if (!c || !out || b < 0 || b >= c->batch || site < 0 || site >= c->n) return TNMPS_ERR_ARG;
  int32_t d[2];
  cudaError_t e = cudaMemcpyAsync(d, c->dims + (size_t)b * (c->n + 1) + site, 8,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "read dims");
  const size_t cnt = (size_t)d[0] * 2 * d[1];
  if (cnt > cap) return fail(c, TNMPS_ERR_ARG, "output capacity too small");
  const size_t esz = c->dtype == TNMPS_C128 ? 16 : 8;
  std::vector<char> buf(cnt * esz);
  const char *src = (const char *)c->sites + esz * ((size_t)b * c->state_elems + c->site_off[site]);
  e = cudaMemcpy(buf.data(), src, cnt * esz, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "read site");
  if (c->dtype == TNMPS_C128) {
    memcpy(out, buf.data(), cnt * 16);
  } else {
    const float *f = (const float *)buf.data();
    for (size_t i = 0; i < 2 * cnt; ++i) out[i] = f[i];
  }
  if (dl) *dl = d[0];
  if (dr) *dr = d[1];
  return TNMPS_OK;
}

int tnmps_get_centre(const tnmps_ctx *c) { return c ? c->centre : -1; }

tnmps_status tnmps_get_stats(tnmps_ctx *c, tnmps_stats *out) {
  if (!c || !out) return TNMPS_ERR_ARG;
  unsigned long long h[CNT_NUM];
  cudaError_t e = cudaMemcpyAsync(h, c->counters, sizeof h, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "read counters");
  out->gates2q = h[CNT_GATES2Q];
  out->gates2q_full = h[CNT_GATES2Q_FULL];
  out->jacobi_pair_rows = h[CNT_PAIR_ROWS];
  out->jacobi_rotations = h[CNT_ROTATIONS];
  out->jacobi_sweeps = h[CNT_SWEEPS];
  out->svds = h[CNT_SVDS];
  out->env_updates = h[CNT_ENV_UPDATES];
  out->env_flops = h[CNT_ENV_FLOPS];
  out->jacobi_rot_rows = h[CNT_ROT_ROWS];
  out->launches = c->launches;
  out->jacobi_alg_bytes = h[CNT_JAC_BYTES];
  return TNMPS_OK;
}

static void prof_drain(tnmps_ctx *c) {
  for (auto &r : c->prof_open) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.cls] += ms;
      c->prof_cnt[r.cls] += 1;
    }
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  c->prof_open.clear();
}

tnmps_status tnmps_profile(tnmps_ctx *c, uint32_t mask) {
  if (!c) return TNMPS_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
  prof_drain(c);
  for (int i = 0; i < PC_NUM; ++i) {
    c->prof_ms[i] = 0;
    c->prof_cnt[i] = 0;
  }
  c->prof_mask = mask;
  return TNMPS_OK;
}

tnmps_status tnmps_profile_read(tnmps_ctx *c, double *ms, uint64_t *count) {
  if (!c) return TNMPS_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
  prof_drain(c);
  for (int i = 0; i < PC_NUM; ++i) {
    if (ms) ms[i] = c->prof_ms[i];
    if (count) count[i] = c->prof_cnt[i];
  }
  return TNMPS_OK;
}

const char *tnmps_last_error(const tnmps_ctx *c) {
  return c ? c->last_error.c_str() : "null context";
}

tnmps_status tnmps_jacobi_svd_dev(tnmps_dtype dtype, int batch, int m, int n, void *a, int lda,
                                  double *sigma, int32_t *sweeps, int max_sweeps, void *stream) {
  if (!valid_dtype(dtype) || batch < 1 || m < 1 || n < 1 || m > TNMPS_JACOBI_MAX_DIM ||
      n > TNMPS_JACOBI_MAX_DIM || lda < m || !a)
    return TNMPS_ERR_ARG;
  cudaError_t e = launch_jacobi_standalone(dtype, batch, m, n, a, lda, sigma, sweeps, max_sweeps,
                                           (cudaStream_t)stream);
  return e == cudaSuccess ? TNMPS_OK : TNMPS_ERR_CUDA;
}

tnmps_status tnmps_set_svd_tolerance(tnmps_ctx *c, double factor) {
  if (!c) return TNMPS_ERR_ARG;
  if (!(factor >= 1.0 && factor <= 4096.0))
    return fail(c, TNMPS_ERR_ARG, "tolerance factor must lie in [1, 4096]");
  c->jacobi_tolfac = (float)factor;
  return TNMPS_OK;
}

tnmps_status tnmps_set_svd_precondition(tnmps_ctx *c, int mode) {
  if (!c) return TNMPS_ERR_ARG;
  if (mode != 0 && mode != 1) return fail(c, TNMPS_ERR_ARG, "svd precondition mode must be 0 or 1");
  c->svd_lq = mode;
  return TNMPS_OK;
}

tnmps_status tnmps_set_tuning(tnmps_ctx *c, const tnmps_tuning *t) {
  if (!c || !t) return TNMPS_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (t->jacobi_shape[k] != 0 && t->jacobi_shape[k] != 1)
      return fail(c, TNMPS_ERR_ARG, "jacobi_shape must be 0 or 1");
  if (t->gemm_stages != 0 && t->gemm_stages != 2 && t->gemm_stages != 3)
    return fail(c, TNMPS_ERR_ARG, "gemm_stages must be 0, 2 or 3");
  if (t->sweep_fused != 0 && t->sweep_fused != 1)
    return fail(c, TNMPS_ERR_ARG, "sweep_fused must be 0 or 1");
  c->tuning = *t;
  return TNMPS_OK;
}

tnmps_status tnmps_get_tuning(const tnmps_ctx *c, tnmps_tuning *t) {
  if (!c || !t) return TNMPS_ERR_ARG;
  *t = c->tuning;
  return TNMPS_OK;
}

tnmps_status tnmps_debug_wait_timeout(tnmps_ctx *c, int64_t max_cycles) {
  if (!c) return TNMPS_ERR_ARG;
  if (max_cycles < 1 || max_cycles > (int64_t)1 << 31)
    return fail(c, TNMPS_ERR_ARG, "max_cycles out of range");
  cudaError_t e = launch_debug_wait(c->err, max_cycles, c->stream);
  ++c->launches;
  if (e != cudaSuccess) return cuda_fail(c, e, "debug wait");
  return TNMPS_OK;
}

tnmps_status tnmps_debug_inject(tnmps_ctx *c, int nth, tnmps_status status) {
  if (!c || nth < 0) return TNMPS_ERR_ARG;
  c->inject_nth = nth > 0 ? c->call_count + nth : 0;
  c->inject_status = status;
  return TNMPS_OK;
}

}  // extern "C"
