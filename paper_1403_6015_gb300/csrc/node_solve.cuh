// The per-node step of the level-by-level factorization (Sec. 3.2): with the half-node
// sums of Phi_j^T Q (Q = the node's rows of the panel and right-hand sides), form
// M = [I, V^T Vt; U^T Ut, I] = I + W L, factor it (LU with partial pivoting), take
// log|det M| (Sylvester's theorem, Sec. 4: det(I + L W) = det(I + W L)), and solve
// Z = M^-1 [V^T P_R; U^T P_L] for the update P_L -= Ut Z_top, P_R -= Vt Z_bot.
#pragma once

#include "ff.cuh"
#include "hodlr_internal.cuh"

namespace hodlr {

struct NodeArgs {
  const double* half;   // per half-node sums, (2^(j+1)) x stride, each r x w row-major
  int64_t stride;
  int j, r, w;          // level, padded rank, partial width
  int cj;               // own columns start (factor mode), -1 in solve mode
  int wz;               // Z width
  double* Mlu;          // level's LU factors, (2r)^2 per node
  int32_t* Mpiv;        // level's pivots, 2r per node
  double* node_logdet;  // per node (level order)
  double* Z;            // level scratch, z_stride = 2 r wz per node
  int64_t z_stride;
  int32_t* flags;
  int zff;              // 1 (mixed form): Z's panel columns (q < cj) as double-float pairs,
                        // its right-hand-side columns FP64; 0: all FP64
  int signed_det;       // 1 (indefinite C): a negative det M toggles kFlagNegDet; 0: it is
                        // an error (kFlagNotSpd)
};

// Record the sign of one block determinant in the device flags.
__device__ __forceinline__ void record_sign(const NodeArgs& a, int sgn) {
  if (sgn == 0 || (sgn < 0 && !a.signed_det)) atomicOr(a.flags, kFlagNotSpd);
  else if (sgn < 0) atomicXor(a.flags, kFlagNegDet);
}

// Partial column of Z column q: ancestors' panel columns keep their index, the right-hand
// sides sit after the node's own r columns in factor mode.
__device__ __forceinline__ int zcol(const NodeArgs& a, int q) {
  return (a.cj >= 0 && q >= a.cj) ? q + a.r : q;
}

// Node k of level a.j, by the whole calling block: M, its LU with partial pivoting and
// log|det| (factor mode) or the stored LU (solve mode), then Z = M^-1 [V^T P_R; U^T P_L].
// M is (2r)^2 doubles of shared memory, piv 2r ints, lds_p / sgn_p two shared scalars.
// The half sums are read through L2 (they may have been written by other blocks of the
// same launch).
static __device__ void node_solve(const NodeArgs& a, int k, bool factor, double* M, int* piv,
                           double* lds_p, int* sgn_p) {
  double& lds = *lds_p;
  int& sgn = *sgn_p;
  int node = (1 << a.j) - 1 + k;
  int r = a.r, m2 = 2 * r, tid = threadIdx.x, nthr = blockDim.x;
  const double* L = a.half + (int64_t)(2 * k) * a.stride;      // U^T (.) over the left half
  const double* Rt = a.half + (int64_t)(2 * k + 1) * a.stride; // V^T (.) over the right half
  double* Mg = a.Mlu + (int64_t)k * m2 * m2;
  int32_t* pg = a.Mpiv + (int64_t)k * m2;
  if (factor) {
    for (int e = tid; e < m2 * m2; e += nthr) {
      int row = e / m2, col = e - row * m2;
      double v;
      if (row < r && col < r) v = row == col ? 1.0 : 0.0;
      else if (row >= r && col >= r) v = row == col ? 1.0 : 0.0;
      else if (row < r) v = __ldcg(Rt + row * a.w + a.cj + (col - r));   // V^T Vt
      else v = __ldcg(L + (row - r) * a.w + a.cj + col);                 // U^T Ut
      M[e] = v;
    }
    __syncthreads();
    if (tid == 0) {
      lds = 0.0;
      sgn = 1;
    }
    for (int c = 0; c < m2; ++c) {
      if (tid == 0) {
        int p = c;
        double best = fabs(M[c * m2 + c]);
        for (int i = c + 1; i < m2; ++i)
          if (fabs(M[i * m2 + c]) > best) {
            best = fabs(M[i * m2 + c]);
            p = i;
          }
        piv[c] = p;
        if (p != c) sgn = -sgn;
      }
      __syncthreads();
      int p = piv[c];
      if (p != c)
        for (int jj = tid; jj < m2; jj += nthr) {
          double t = M[c * m2 + jj];
          M[c * m2 + jj] = M[p * m2 + jj];
          M[p * m2 + jj] = t;
        }
      __syncthreads();
      double d = M[c * m2 + c];
      if (tid == 0) {
        if (d == 0.0) sgn = 0;
        else {
          if (d < 0) sgn = -sgn;
          lds += log(fabs(d));
        }
      }
      for (int i = c + 1 + tid; i < m2; i += nthr) {
        double l = d != 0.0 ? M[i * m2 + c] / d : 0.0;
        M[i * m2 + c] = l;
        for (int jj = c + 1; jj < m2; ++jj) M[i * m2 + jj] -= l * M[c * m2 + jj];
      }
      __syncthreads();
    }
    for (int e = tid; e < m2 * m2; e += nthr) Mg[e] = M[e];
    for (int e = tid; e < m2; e += nthr) pg[e] = piv[e];
    if (tid == 0) {
      a.node_logdet[node] = lds;
      record_sign(a, sgn);
    }
  } else {
    for (int e = tid; e < m2 * m2; e += nthr) M[e] = Mg[e];
    for (int e = tid; e < m2; e += nthr) piv[e] = pg[e];
  }
  __syncthreads();
  // Z = M^-1 [V^T P_R; U^T P_L], one thread per column
  double* Zn = a.Z + (int64_t)k * a.z_stride;
  for (int q = tid; q < a.wz; q += nthr) {
    int pc = zcol(a, q);
    for (int row = 0; row < r; ++row) {
      Zn[row * a.wz + q] = __ldcg(Rt + row * a.w + pc);
      Zn[(r + row) * a.wz + q] = __ldcg(L + row * a.w + pc);
    }
    for (int c = 0; c < m2; ++c) {
      int p = piv[c];
      if (p != c) {
        double t = Zn[c * a.wz + q];
        Zn[c * a.wz + q] = Zn[p * a.wz + q];
        Zn[p * a.wz + q] = t;
      }
    }
    for (int i = 1; i < m2; ++i) {
      double s = Zn[i * a.wz + q];
      for (int c = 0; c < i; ++c) s -= M[i * m2 + c] * Zn[c * a.wz + q];
      Zn[i * a.wz + q] = s;
    }
    for (int i = m2 - 1; i >= 0; --i) {
      double s = Zn[i * a.wz + q];
      for (int c = i + 1; c < m2; ++c) s -= M[i * m2 + c] * Zn[c * a.wz + q];
      Zn[i * a.wz + q] = s / M[i * m2 + i];
    }
    if (a.zff && q < a.cj)  // a panel column, in place: this thread owns column q
      for (int i = 0; i < m2; ++i)
        reinterpret_cast<ff*>(Zn)[i * a.wz + q] = ff_from_double(Zn[i * a.wz + q]);
  }
}


}  // namespace hodlr
