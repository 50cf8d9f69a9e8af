// Per-state construction of fused gate matrices on the device (FP64).
//
// The circuit planner folds every run of single-qubit gates into the next
// two-qubit gate on the same site (or into a standalone single-qubit op), so
// the paper's "contract the gate tensor into the MPS" step (Sec. IV) for 1q
// gates costs no extra pass over the site tensors. Parameterised rotations
// are evaluated here from the state's own parameter row.
#pragma once
#include "tnmps_internal.h"

__device__ __forceinline__ void fac_matrix(const Fac1 &f, const double *theta, cx<double> U[4]) {
  if (f.kind == 0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) U[e] = mkc<double>(f.m[2 * e], f.m[2 * e + 1]);
    return;
  }
  double a = f.angle;
  if (f.param >= 0) a += f.scale * theta[f.param];
  double s, c;
  sincos(0.5 * a, &s, &c);
  if (f.kind == 1) {  // RX = [[c, -is], [-is, c]]
    U[0] = mkc<double>(c, 0);
    U[1] = mkc<double>(0, -s);
    U[2] = mkc<double>(0, -s);
    U[3] = mkc<double>(c, 0);
  } else if (f.kind == 2) {  // RY = [[c, -s], [s, c]]
    U[0] = mkc<double>(c, 0);
    U[1] = mkc<double>(-s, 0);
    U[2] = mkc<double>(s, 0);
    U[3] = mkc<double>(c, 0);
  } else {  // RZ = diag(e^{-ia/2}, e^{ia/2})
    U[0] = mkc<double>(c, -s);
    U[1] = mkc<double>(0, 0);
    U[2] = mkc<double>(0, 0);
    U[3] = mkc<double>(c, s);
  }
}

// U = f_{n-1} ... f_0 (factors applied in list order)
__device__ __forceinline__ void side_matrix(const Fac1 *f, int nf, const double *theta,
                                            cx<double> U[4]) {
  U[0] = mkc<double>(1, 0);
  U[1] = mkc<double>(0, 0);
  U[2] = mkc<double>(0, 0);
  U[3] = mkc<double>(1, 0);
  for (int i = 0; i < nf; ++i) {
    cx<double> F[4], T[4];
    fac_matrix(f[i], theta, F);
    T[0] = cadd(cmul(F[0], U[0]), cmul(F[1], U[2]));
    T[1] = cadd(cmul(F[0], U[1]), cmul(F[1], U[3]));
    T[2] = cadd(cmul(F[2], U[0]), cmul(F[3], U[2]));
    T[3] = cadd(cmul(F[2], U[1]), cmul(F[3], U[3]));
#pragma unroll
    for (int e = 0; e < 4; ++e) U[e] = T[e];
  }
}

// G = core * (Ul (x) Ur), basis index 2*s_l + s_r, row-major 4x4.
__device__ __forceinline__ void op2_matrix(const Op2 &op, const double *theta, cx<double> G[16]) {
  cx<double> Ul[4], Ur[4];
  side_matrix(op.fl, op.nl, theta, Ul);
  side_matrix(op.fr, op.nr, theta, Ur);
  cx<double> K[16];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      K[4 * r + c] = cmul(Ul[2 * (r >> 1) + (c >> 1)], Ur[2 * (r & 1) + (c & 1)]);
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      cx<double> acc = mkc<double>(0, 0);
      for (int k = 0; k < 4; ++k)
        acc = cadd(acc, cmul(mkc<double>(op.core[2 * (4 * r + k)], op.core[2 * (4 * r + k) + 1]),
                             K[4 * k + c]));
      G[4 * r + c] = acc;
    }
}

// Same as op2_matrix with the parts given separately (core 4x4 as 32
// doubles, left and right factor lists).
__device__ __forceinline__ void op2_matrix_parts(const double *core, const Fac1 *fl, int nl,
                                                 const Fac1 *fr, int nr, const double *theta,
                                                 cx<double> G[16]) {
  cx<double> Ul[4], Ur[4];
  side_matrix(fl, nl, theta, Ul);
  side_matrix(fr, nr, theta, Ur);
  cx<double> K[16];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c)
      K[4 * r + c] = cmul(Ul[2 * (r >> 1) + (c >> 1)], Ur[2 * (r & 1) + (c & 1)]);
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      cx<double> acc = mkc<double>(0, 0);
      for (int k = 0; k < 4; ++k)
        acc = cadd(acc, cmul(mkc<double>(core[2 * (4 * r + k)], core[2 * (4 * r + k) + 1]),
                             K[4 * k + c]));
      G[4 * r + c] = acc;
    }
}
