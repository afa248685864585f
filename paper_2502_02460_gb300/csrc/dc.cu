// Tridiagonal eigensolver ("Solve" in Table 1): divide and conquer on the real symmetric
// tridiagonal T = (d, e), eigenvalues of all of T and eigenvectors of the k lowest.
//
//  * Tearing (Cuppen): at every split m (between rows m-1 and m) with rho = e[m-1]:
//      T = diag(T1 - |rho| e_last e_last^T, T2 - |rho| e_1 e_1^T) + |rho| u u^T,
//      u = e_{m-1} + sign(rho) e_m.
//  * Leaves (<= 32 rows): implicit QL with shifts, one block per leaf.
//  * Merge of two solved children T1' = Q1 D1 Q1^T, T2' = Q2 D2 Q2^T:
//      T' = Q (D + r zz^T) Q^T,  z = [last row of Q1, sign(rho) first row of Q2] / sqrt(2),
//      r = 2|rho|.  The poles (children eigenvalues, each list sorted) are merged by rank;
//      deflation (|r z_i| <= tol, or two poles so close that a Givens rotation zeroing one
//      z-component leaves an off-diagonal <= tol) is one sequential scan; the K remaining roots of
//      the secular equation 1 + r sum z_i^2/(delta_i - lambda) = 0 are found one per thread in
//      coordinates shifted to the nearest pole, by a bracketed two-pole rational iteration; z is
//      recomputed from the roots (Gu-Eisenstat) so the eigenvectors u_j = z_i/(delta_i - lambda_j)
//      are numerically orthogonal; the new eigenvectors Q u_j come from two GEMMs that use the
//      block structure (columns that live in the top child only, in both, in the bottom only).
//  * Columns are never physically sorted: colmap[a + p] gives the physical column of the p-th
//    smallest eigenvalue of the node starting at a.  At the top merge only the k lowest
//    eigenvectors are formed.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace gev {

namespace {

constexpr int LEAF = 32;
constexpr double EPS = 2.220446049250313e-16;

struct Node {
  int a, m, c;       // rows [a, c), split at m
  int K;             // non-deflated count
  int K1, K2, K3;    // top-only / mixed / bottom-only among the non-deflated
  int ndefl;         // deflated count
  int nrot;          // Givens rotations applied
  int Kout;          // eigenvectors to form (roots with final position < kcut)
  int Dout;          // deflated vectors with final position < kcut
  double r;          // 2|rho|
  double zn2;        // sum of squared non-deflated z
};

// per-level device arrays carved from the D&C workspace, each of length n (indexed by row range)
struct DcArrays {
  double* dsort;   // merged sorted poles
  double* zs;      // z in sorted order
  int* csrc;       // physical column of each sorted entry
  int* tb;         // bit 1: has rows in the top child, bit 2: in the bottom child
  double* nd_d;    // non-deflated poles (ascending)
  double* nd_z;    // their z
  int* nd_col;     // their physical columns
  int* nd_g;       // gather slot (type order) of each non-deflated entry
  double* df_d;    // deflated eigenvalues (ascending after the sort)
  int* df_col;     // their physical columns
  double* mu;      // root offsets
  int* org;        // root origins (index into nd list)
  double* zp;      // recomputed z
  int* pos_r;      // final position of each root within the node
  int* pos_d;      // final position of each deflated entry
  int* rot_p;      // rotations: column pairs and (c, s)
  int* rot_i;
  double* rot_c;
  double* rot_s;
  int* colmap;     // physical column of each sorted position
  int* colmap2;
  double* dwork;   // torn diagonal
  Node* nodes;     // per-level node descriptors (device)
};

// ------------------------------------------------------------------------------------ tearing --
__global__ void k_tear(int n, int nleaf, const double* d, const double* e, double* dw) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dw[i] = d[i];
  __syncthreads();
}
__global__ void k_tear2(int n, int nleaf, const double* e, double* dw) {
  // boundary of leaf q (q = 1 .. nleaf-1) at row floor(q n / nleaf)
  for (int q = 1 + blockIdx.x * blockDim.x + threadIdx.x; q < nleaf; q += gridDim.x * blockDim.x) {
    const int m = (int)(((long long)q * n) / nleaf);
    const double rho = fabs(e[m - 1]);
    dw[m - 1] -= rho;
    dw[m] -= rho;
  }
}

// ------------------------------------------------------------------------------------- leaves --
// Implicit QL on the leaf (rows [a, a+sz)), eigenvectors accumulated in shared memory; thread 0
// runs the scalar recurrence and records each sweep's rotations, all threads apply them.
__global__ void __launch_bounds__(64) k_leaf(int n, int nleaf, const double* dw, const double* e,
                                             double* w, double* Q, long long ldq, int* colmap,
                                             int* status) {
  __shared__ double Z[LEAF][LEAF + 1];
  __shared__ double dd[LEAF], ee[LEAF];
  __shared__ double rc[LEAF], rs[LEAF];
  __shared__ int ri[LEAF];
  __shared__ int nrot, done, fail;
  __shared__ int perm[LEAF];
  const int q = blockIdx.x;
  const int a = (int)(((long long)q * n) / nleaf);
  const int c = (int)(((long long)(q + 1) * n) / nleaf);
  const int sz = c - a;
  const int tid = threadIdx.x;
  for (int i = tid; i < sz; i += blockDim.x) {
    dd[i] = dw[a + i];
    ee[i] = (i + 1 < sz) ? e[a + i] : 0.0;
    for (int j = 0; j < sz; ++j) Z[i][j] = (i == j) ? 1.0 : 0.0;
  }
  if (tid == 0) { done = 0; fail = 0; }
  __syncthreads();
  // thread-0 state of the QL iteration
  int l = 0, iter = 0, total = 0;
  while (true) {
    if (tid == 0) {
      nrot = 0;
      // advance to the next sweep to perform (or finish)
      while (true) {
        if (l >= sz) { done = 1; break; }
        int m = l;
        while (m + 1 < sz) {
          const double dsum = fabs(dd[m]) + fabs(dd[m + 1]);
          if (fabs(ee[m]) <= EPS * dsum) break;
          ++m;
        }
        if (m == l) { ++l; iter = 0; continue; }
        if (++total > 30 * sz) { fail = 1; done = 1; break; }
        ++iter;
        double g = (dd[l + 1] - dd[l]) / (2.0 * ee[l]);
        double r = hypot(g, 1.0);
        g = dd[m] - dd[l] + ee[l] / (g + copysign(r, g));
        double s = 1.0, cc = 1.0, p = 0.0;
        bool early = false;
        for (int i = m - 1; i >= l; --i) {
          const double f = s * ee[i], b = cc * ee[i];
          r = hypot(f, g);
          ee[i + 1] = r;
          if (r == 0.0) { dd[i + 1] -= p; ee[m] = 0.0; early = true; break; }
          s = f / r;
          cc = g / r;
          g = dd[i + 1] - p;
          r = (dd[i] - g) * s + 2.0 * cc * b;
          p = s * r;
          dd[i + 1] = g + p;
          g = cc * r - b;
          ri[nrot] = i; rc[nrot] = cc; rs[nrot] = s; ++nrot;
        }
        if (!early) { dd[l] -= p; ee[l] = g; ee[m] = 0.0; }
        break;  // one sweep recorded
      }
    }
    __syncthreads();
    const int nr = nrot;
    for (int row = tid; row < sz; row += blockDim.x) {
      for (int t = 0; t < nr; ++t) {
        const int i = ri[t];
        const double zi = Z[row][i], zi1 = Z[row][i + 1];
        Z[row][i + 1] = rs[t] * zi + rc[t] * zi1;
        Z[row][i] = rc[t] * zi - rs[t] * zi1;
      }
    }
    __syncthreads();
    if (done) break;
  }
  if (tid == 0) {
    if (fail) atomicCAS(&status[ST_NOCONV], 0, 301);
    for (int i = 0; i < sz; ++i) perm[i] = i;
    for (int i = 1; i < sz; ++i) {  // stable insertion sort of eigenvalue indices
      int pi = perm[i];
      int j = i - 1;
      while (j >= 0 && dd[perm[j]] > dd[pi]) { perm[j + 1] = perm[j]; --j; }
      perm[j + 1] = pi;
    }
  }
  __syncthreads();
  for (int i = tid; i < sz; i += blockDim.x) {
    w[a + i] = dd[perm[i]];
    colmap[a + i] = a + i;
    for (int j = 0; j < sz; ++j) Q[(a + j) + (long long)(a + i) * ldq] = Z[j][perm[i]];
  }
}

// ------------------------------------------------------------------------------ merge: prepare --
// One block per node: z, rank merge of the two sorted pole lists, deflation scan (thread 0),
// rotations applied to the physical columns, sort of the deflated list, gather order by type.
__global__ void __launch_bounds__(1024) k_merge_prep(int n, Node* nodes, const double* e,
                                                      const double* w, double* Q, long long ldq,
                                                      DcArrays A) {
  Node& nd = nodes[blockIdx.x];
  const int a = nd.a, m = nd.m, c = nd.c;
  const int n1 = m - a, nn = c - a;
  const int tid = threadIdx.x, NTH = blockDim.x;
  const double rho = e[m - 1];
  const double sg = rho < 0 ? -1.0 : 1.0;
  const double r = 2.0 * fabs(rho);
  const double isq2 = 0.70710678118654752440;
  // rank merge: child 1 = w[a .. m), child 2 = w[m .. c), both ascending
  for (int i = tid; i < nn; i += NTH) {
    double di;
    int pos, col;
    double zi;
    int tbits;
    if (i < n1) {
      di = w[a + i];
      // number of child-2 entries strictly below di
      int lo = 0, hi = nn - n1;
      while (lo < hi) { int md = (lo + hi) >> 1; if (w[m + md] < di) lo = md + 1; else hi = md; }
      pos = i + lo;
      col = A.colmap[a + i];
      zi = Q[(m - 1) + (long long)col * ldq] * isq2;
      tbits = 1;
    } else {
      const int j = i - n1;
      di = w[m + j];
      int lo = 0, hi = n1;  // child-1 entries <= di
      while (lo < hi) { int md = (lo + hi) >> 1; if (w[a + md] <= di) lo = md + 1; else hi = md; }
      pos = j + lo;
      col = A.colmap[m + j];
      zi = sg * Q[m + (long long)col * ldq] * isq2;
      tbits = 2;
    }
    A.dsort[a + pos] = di;
    A.zs[a + pos] = zi;
    A.csrc[a + pos] = col;
    A.tb[a + pos] = tbits;
  }
  __syncthreads();
  __shared__ int sK, sD, sR;
  if (tid == 0) {
    const double dmax = fmax(fabs(A.dsort[a]), fabs(A.dsort[c - 1]));
    const double tol = 8.0 * EPS * fmax(dmax, r);
    int K = 0, D = 0, R = 0;
    int prev = -1;  // sorted index of the pending non-deflated candidate
    double zn2 = 0.0;
    for (int i = 0; i < nn; ++i) {
      const int ii = a + i;
      const double zi = A.zs[ii];
      if (r * fabs(zi) <= tol) {  // negligible coupling: eigenpair kept as is
        A.df_d[a + D] = A.dsort[ii];
        A.df_col[a + D] = A.csrc[ii];
        ++D;
        continue;
      }
      if (prev >= 0) {
        const int pj = a + prev;
        const double zp = A.zs[pj];
        const double tau = hypot(zp, zi);
        const double cs = zi / tau, sn = zp / tau;
        const double dp = A.dsort[pj], di = A.dsort[ii];
        if (fabs((di - dp) * cs * sn) <= tol) {
          // rotate the pair so z_prev = 0: prev deflates
          A.zs[ii] = tau;
          A.zs[pj] = 0.0;
          A.dsort[pj] = cs * cs * dp + sn * sn * di;
          A.dsort[ii] = sn * sn * dp + cs * cs * di;
          const int cp = A.csrc[pj], ci = A.csrc[ii];
          A.rot_p[a + R] = cp;
          A.rot_i[a + R] = ci;
          A.rot_c[a + R] = cs;
          A.rot_s[a + R] = sn;
          ++R;
          const int u = A.tb[pj] | A.tb[ii];
          A.tb[pj] = u;
          A.tb[ii] = u;
          A.df_d[a + D] = A.dsort[pj];
          A.df_col[a + D] = cp;
          ++D;
          prev = i;
          continue;
        }
        // prev is final
        A.nd_d[a + K] = dp;
        A.nd_z[a + K] = zp;
        A.nd_col[a + K] = A.csrc[pj];
        A.nd_g[a + K] = A.tb[pj];  // temporarily the type bits
        zn2 += zp * zp;
        ++K;
      }
      prev = i;
    }
    if (prev >= 0) {
      const int pj = a + prev;
      A.nd_d[a + K] = A.dsort[pj];
      A.nd_z[a + K] = A.zs[pj];
      A.nd_col[a + K] = A.csrc[pj];
      A.nd_g[a + K] = A.tb[pj];
      zn2 += A.zs[pj] * A.zs[pj];
      ++K;
    }
    // stable insertion sort of the deflated list (rotations perturb its order only locally)
    for (int i = 1; i < D; ++i) {
      const double dv = A.df_d[a + i];
      const int cv = A.df_col[a + i];
      int j = i - 1;
      while (j >= 0 && A.df_d[a + j] > dv) {
        A.df_d[a + j + 1] = A.df_d[a + j];
        A.df_col[a + j + 1] = A.df_col[a + j];
        --j;
      }
      A.df_d[a + j + 1] = dv;
      A.df_col[a + j + 1] = cv;
    }
    // gather order: top-only, mixed, bottom-only
    int K1 = 0, K2 = 0, K3 = 0;
    for (int i = 0; i < K; ++i) {
      const int t = A.nd_g[a + i];
      if (t == 1) ++K1; else if (t == 3) ++K2; else ++K3;
    }
    int c1 = 0, c2 = K1, c3 = K1 + K2;
    for (int i = 0; i < K; ++i) {
      const int t = A.nd_g[a + i];
      A.nd_g[a + i] = (t == 1) ? c1++ : (t == 3 ? c2++ : c3++);
    }
    nd.K = K; nd.K1 = K1; nd.K2 = K2; nd.K3 = K3; nd.ndefl = D; nd.nrot = R;
    nd.r = r; nd.zn2 = zn2;
    nd.Kout = K; nd.Dout = D;
    sK = K; sD = D; sR = R;
  }
  __syncthreads();
  // apply the rotations, in order, to the physical columns (rows a .. c-1)
  const int R = sR;
  for (int t = 0; t < R; ++t) {
    const int cp = A.rot_p[a + t], ci = A.rot_i[a + t];
    const double cs = A.rot_c[a + t], sn = A.rot_s[a + t];
    for (int row = a + tid; row < c; row += NTH) {
      const double qp = Q[row + (long long)cp * ldq], qi = Q[row + (long long)ci * ldq];
      Q[row + (long long)cp * ldq] = cs * qp - sn * qi;
      Q[row + (long long)ci * ldq] = sn * qp + cs * qi;
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------- merge: secular --
// The secular function and its pieces at mu, by one warp: lane l sums the poles l, l + 32, ...; the
// partial sums are reduced to lane 0 in a fixed order and broadcast, so every lane holds the same bits
// (the root iteration below branches on them identically in all lanes).
__device__ void eval_secular(int K, int j, int o, const double* delta, const double* z, double r,
                             double mu, double& f, double& psi, double& dpsi, double& phi,
                             double& dphi) {
  const int lane = threadIdx.x & 31;
  const double dO = delta[o];
  double a = 0.0, b = 0.0, c = 0.0, e = 0.0;
  for (int i = lane; i < K; i += 32) {
    const double di = (delta[i] - dO) - mu;
    const double zi = z[i];
    const double t = zi / di;
    if (i <= j) { a += zi * t; b += t * t; }
    else { c += zi * t; e += t * t; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
    c += __shfl_down_sync(0xffffffffu, c, off);
    e += __shfl_down_sync(0xffffffffu, e, off);
  }
  psi = __shfl_sync(0xffffffffu, a, 0);
  dpsi = __shfl_sync(0xffffffffu, b, 0);
  phi = __shfl_sync(0xffffffffu, c, 0);
  dphi = __shfl_sync(0xffffffffu, e, 0);
  f = 1.0 + r * (psi + phi);
}

// One warp per root (blockDim 256: 8 roots per block); lane 0 writes the result.
__global__ void __launch_bounds__(256) k_secular(Node* nodes, DcArrays A, int* status) {
  const Node nd = nodes[blockIdx.y];
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const bool lead = (threadIdx.x & 31) == 0;
  const int K = nd.K;
  if (j >= K) return;  // uniform per warp
  const int a = nd.a;
  const double* delta = A.nd_d + a;
  const double* z = A.nd_z + a;
  const double r = nd.r;
  int o;
  double lo, hi;
  const bool last = (j == K - 1);
  if (!last) {
    const double gap = delta[j + 1] - delta[j];
    const double mid = 0.5 * gap;
    double f, psi, dpsi, phi, dphi;
    eval_secular(K, j, j, delta, z, r, mid, f, psi, dpsi, phi, dphi);
    if (f >= 0.0) { o = j; lo = 0.0; hi = mid; }
    else { o = j + 1; lo = -mid; hi = 0.0; }
  } else {
    o = j;
    lo = 0.0;
    hi = r * nd.zn2;
  }
  const double dO = delta[o];
  const double D1b = delta[j] - dO;                       // left pole of the interval (shifted)
  const double D2b = last ? 0.0 : delta[j + 1] - dO;      // right pole (unused for the last root)
  double mu = 0.5 * (lo + hi);
  bool conv = false;
  for (int it = 0; it < 200; ++it) {
    double f, psi, dpsi, phi, dphi;
    eval_secular(K, j, o, delta, z, r, mu, f, psi, dpsi, phi, dphi);
    if (f == 0.0) { conv = true; break; }
    if (f < 0.0) lo = mu; else hi = mu;
    const double errb = 8.0 * EPS * (double)(K + 2) * (1.0 + r * (fabs(psi) + fabs(phi)));
    if (fabs(f) <= errb) { conv = true; break; }
    if (hi - lo <= 4.0 * EPS * fmax(fabs(lo), fabs(hi))) { conv = true; break; }
    // two-pole rational model g(x) = a + q/(D1 - eta) + Q/(D2 - eta), eta = x - mu
    double eta;
    const double D1 = D1b - mu;
    const double q = r * dpsi * D1 * D1;
    if (!last) {
      const double D2 = D2b - mu;
      const double Qc = r * dphi * D2 * D2;
      const double aa = f - q / D1 - Qc / D2;
      const double c0 = D1 * D2 * f;
      const double b0 = aa * (D1 + D2) + q + Qc;
      if (aa == 0.0) {
        eta = c0 / b0;
      } else {
        double disc = b0 * b0 - 4.0 * aa * c0;
        disc = disc > 0.0 ? sqrt(disc) : 0.0;
        double e1, e2;
        if (b0 >= 0.0) { e1 = (b0 + disc) / (2.0 * aa); e2 = 2.0 * c0 / (b0 + disc); }
        else { e1 = (b0 - disc) / (2.0 * aa); e2 = 2.0 * c0 / (b0 - disc); }
        const bool in1 = (mu + e1 > lo) && (mu + e1 < hi);
        const bool in2 = (mu + e2 > lo) && (mu + e2 < hi);
        eta = in2 ? e2 : (in1 ? e1 : 0.5 * (lo + hi) - mu);
      }
    } else {
      const double aa = f - q / D1;
      eta = (aa != 0.0) ? D1 + q / aa : 0.5 * (lo + hi) - mu;
    }
    double mnew = mu + eta;
    const bool ok = last ? (mnew > lo && mnew <= hi) : (mnew > lo && mnew < hi);
    if (!ok || !(mnew == mnew)) mnew = 0.5 * (lo + hi);
    if (fabs(mnew - mu) <= 2.0 * EPS * fabs(mnew)) { mu = mnew; conv = true; break; }
    mu = mnew;
  }
  if (!lead) return;
  if (!conv) atomicCAS(&status[ST_NOCONV], 0, 302);
  A.mu[a + j] = mu;
  A.org[a + j] = o;
}

// Gu-Eisenstat: z'_i^2 = prod_j (lambda_j - delta_i) / (r prod_{j != i} (delta_j - delta_i)).
__global__ void k_zprime(Node* nodes, DcArrays A) {
  const Node nd = nodes[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = nd.K;
  if (i >= K) return;
  const int a = nd.a;
  const double* delta = A.nd_d + a;
  const double* mu = A.mu + a;
  const int* org = A.org + a;
  const double di = delta[i];
  auto lam_minus = [&](int j) { return (delta[org[j]] - di) + mu[j]; };
  double prod = lam_minus(K - 1) / nd.r;
  for (int j = 0; j < i; ++j) prod *= lam_minus(j) / (delta[j] - di);
  for (int j = i; j < K - 1; ++j) prod *= lam_minus(j) / (delta[j + 1] - di);
  const double zi = A.nd_z[a + i];
  A.zp[a + i] = copysign(sqrt(fabs(prod)), zi);
}

// Final positions of roots and deflated entries within each node; eigenvalues in sorted order.
__global__ void k_positions(Node* nodes, DcArrays A, int kcut, int* status) {
  Node& nd = nodes[blockIdx.y];
  const int a = nd.a, K = nd.K, D = nd.ndefl;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < K + D; t += gridDim.x * blockDim.x) {
    if (t < K) {
      const double lam = A.nd_d[a + A.org[a + t]] + A.mu[a + t];
      int lo = 0, hi = D;
      while (lo < hi) { int md = (lo + hi) >> 1; if (A.df_d[a + md] < lam) lo = md + 1; else hi = md; }
      A.pos_r[a + t] = t + lo;
    } else {
      const int u = t - K;
      const double dv = A.df_d[a + u];
      int lo = 0, hi = K;
      while (lo < hi) {
        int md = (lo + hi) >> 1;
        const double lam = A.nd_d[a + A.org[a + md]] + A.mu[a + md];
        if (lam <= dv) lo = md + 1; else hi = md;
      }
      A.pos_d[a + u] = u + lo;
    }
  }
}

// Count the roots / deflated entries whose position is below kcut (prefixes: positions increase).
__global__ void k_count_out(Node* nodes, DcArrays A, int kcut) {
  Node& nd = nodes[blockIdx.x];
  if (threadIdx.x != 0) return;
  const int a = nd.a;
  int ko = 0, dout = 0;
  for (int t = 0; t < nd.K; ++t) if (A.pos_r[a + t] < kcut) ++ko;
  for (int u = 0; u < nd.ndefl; ++u) if (A.pos_d[a + u] < kcut) ++dout;
  nd.Kout = ko;
  nd.Dout = dout;
}

// U (gather order rows x Kout, ld ldu) column j: u_i = z'_i/(delta_i - lambda_j), normalised.
__global__ void k_vectors(Node* nodes, DcArrays A, double* U, long long ldu) {
  const Node nd = nodes[blockIdx.y];
  const int j = blockIdx.x;
  if (j >= nd.Kout) return;
  const int a = nd.a, K = nd.K;
  const double* delta = A.nd_d + a;
  const double dO = delta[A.org[a + j]];
  const double mu = A.mu[a + j];
  double* col = U + (long long)(a + j) * ldu;  // rows 0 .. K-1 of column a + j
  double ss = 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const double v = A.zp[a + i] / ((delta[i] - dO) - mu);
    col[A.nd_g[a + i]] = v;
    ss += v * v;
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    red[0] = 1.0 / sqrt(t);
  }
  __syncthreads();
  const double inv = red[0];
  for (int i = threadIdx.x; i < K; i += blockDim.x) col[i] *= inv;
}

// Qg[:, a + g] = Q[:, nd_col] (rows a .. c-1) in gather order; deflated columns (position < kcut)
// go straight to Qout[:, a + K + u].
__global__ void k_gather(Node* nodes, DcArrays A, const double* Q, long long ldq, double* Qg,
                         double* Qout) {
  const Node nd = nodes[blockIdx.y];
  const int a = nd.a, c = nd.c, nn = c - a;
  const int t = blockIdx.x;
  if (t < nd.K) {
    const int src = A.nd_col[a + t];
    const int g = A.nd_g[a + t];
    for (int i = threadIdx.x; i < nn; i += blockDim.x)
      Qg[(a + i) + (long long)(a + g) * ldq] = Q[(a + i) + (long long)src * ldq];
  } else if (t < nd.K + nd.ndefl) {
    const int u = t - nd.K;
    if (A.pos_d[a + u] >= 0x7fffffff) return;
    const int src = A.df_col[a + u];
    for (int i = threadIdx.x; i < nn; i += blockDim.x)
      Qout[(a + i) + (long long)(a + nd.K + u) * ldq] = Q[(a + i) + (long long)src * ldq];
  }
}

// Sorted eigenvalues and the column map of the merged node.
__global__ void k_finalize(Node* nodes, DcArrays A, double* w) {
  const Node nd = nodes[blockIdx.y];
  const int a = nd.a, K = nd.K, D = nd.ndefl;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < K + D; t += gridDim.x * blockDim.x) {
    if (t < K) {
      const int p = A.pos_r[a + t];
      w[a + p] = A.nd_d[a + A.org[a + t]] + A.mu[a + t];
      A.colmap2[a + p] = a + t;
    } else {
      const int u = t - K;
      const int p = A.pos_d[a + u];
      w[a + p] = A.df_d[a + u];
      A.colmap2[a + p] = a + K + u;
    }
  }
}

__global__ void k_copy_int(int n, const int* src, int* dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

// Z[:, p] = Q[:, colmap[p]] for p < k (rows 0 .. n-1).
__global__ void k_output(int n, int k, const double* Q, long long ldq, const int* colmap, double* Z,
                         long long ldz) {
  const int p = blockIdx.x;
  if (p >= k) return;
  const int src = colmap[p];
  for (int i = threadIdx.x; i < n; i += blockDim.x) Z[i + (long long)p * ldz] = Q[i + (long long)src * ldq];
}

}  // namespace

int stedc(Sys& s, const double* d, const double* e, int k, double* w, double* Z, int ldz, int* deflated) {
  const int n = s.n;
  cudaStream_t st = s.stream;
  // carve the workspace
  char* p = (char*)s.dcws;
  auto take = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return (void*)r;
  };
  DcArrays A;
  const size_t nd8 = sizeof(double) * (size_t)n, ni4 = sizeof(int) * (size_t)n;
  A.dsort = (double*)take(nd8); A.zs = (double*)take(nd8); A.csrc = (int*)take(ni4); A.tb = (int*)take(ni4);
  A.nd_d = (double*)take(nd8); A.nd_z = (double*)take(nd8); A.nd_col = (int*)take(ni4); A.nd_g = (int*)take(ni4);
  A.df_d = (double*)take(nd8); A.df_col = (int*)take(ni4); A.mu = (double*)take(nd8); A.org = (int*)take(ni4);
  A.zp = (double*)take(nd8); A.pos_r = (int*)take(ni4); A.pos_d = (int*)take(ni4);
  A.rot_p = (int*)take(ni4); A.rot_i = (int*)take(ni4); A.rot_c = (double*)take(nd8); A.rot_s = (double*)take(nd8);
  A.colmap = (int*)take(ni4); A.colmap2 = (int*)take(ni4); A.dwork = (double*)take(nd8);
  A.nodes = (Node*)take(sizeof(Node) * (size_t)(n / 2 + 2));
  if ((size_t)(p - (char*)s.dcws) > s.dcws_bytes) return GEV_ERR_OOM;

  double* Qa = s.Q;
  double* Qb = s.Q2;
  double* Qg = (double*)s.W1;
  double* U = (double*)s.Yk;  // s.A keeps the FP64 standard matrix (mixed-form refinement)
  const long long ldq = n;

  // Every column of a node must be zero outside the node's rows (block-diagonal eigenvector
  // matrices): deflated columns are copied over the whole node range and Givens rotations mix full
  // columns.  Both buffers are cleared here, so rows a level never writes stay zero.
  GEV_CUDA_TRY(cudaMemsetAsync(Qa, 0, sizeof(double) * (size_t)n * n, st));
  GEV_CUDA_TRY(cudaMemsetAsync(Qb, 0, sizeof(double) * (size_t)n * n, st));
  int nleaf = 1;
  while ((n + nleaf - 1) / nleaf > LEAF) nleaf *= 2;
  const unsigned eb = cdiv(n, 256) < 1024u ? cdiv(n, 256) : 1024u;
  GEV_COUNT(s);
  k_tear<<<eb, 256, 0, st>>>(n, nleaf, d, e, A.dwork);
  if (nleaf > 1) {
    GEV_COUNT(s);
    k_tear2<<<cdiv(nleaf, 256), 256, 0, st>>>(n, nleaf, e, A.dwork);
  }
  GEV_COUNT(s);
  k_leaf<<<nleaf, 64, 0, st>>>(n, nleaf, A.dwork, e, w, Qa, ldq, A.colmap, s.status);
  GEV_TRY(last_error());

  std::vector<Node> hn;
  int top_deflated = 0;
  for (int span = 2; span <= nleaf; span *= 2) {
    const int nnodes = nleaf / span;
    const bool top = (span == nleaf);
    hn.assign(nnodes, Node{});
    for (int q = 0; q < nnodes; ++q) {
      hn[q].a = (int)(((long long)q * span * n) / nleaf);
      hn[q].m = (int)(((long long)(q * span + span / 2) * n) / nleaf);
      hn[q].c = (int)(((long long)(q + 1) * span * n) / nleaf);
    }
    GEV_CUDA_TRY(cudaMemcpyAsync(A.nodes, hn.data(), sizeof(Node) * nnodes, cudaMemcpyHostToDevice, st));
    GEV_COUNT(s);
    k_merge_prep<<<nnodes, 1024, 0, st>>>(n, A.nodes, e, w, Qa, ldq, A);
    GEV_TRY(last_error());
    GEV_CUDA_TRY(cudaMemcpyAsync(hn.data(), A.nodes, sizeof(Node) * nnodes, cudaMemcpyDeviceToHost, st));
    GEV_CUDA_TRY(cudaStreamSynchronize(st));
    int Kmax = 0, Tmax = 0;
    for (auto& x : hn) {
      Kmax = std::max(Kmax, x.K);
      Tmax = std::max(Tmax, x.K + x.ndefl);
    }
    if (Kmax > 0) {
      GEV_COUNT(s);
      k_secular<<<dim3(cdiv(Kmax, 8), nnodes), 256, 0, st>>>(A.nodes, A, s.status);
      GEV_COUNT(s);
      k_zprime<<<dim3(cdiv(Kmax, 128), nnodes), 128, 0, st>>>(A.nodes, A);
    }
    const int kcut = top ? k : 0x7fffffff;
    GEV_COUNT(s);
    k_positions<<<dim3(cdiv(Tmax, 256), nnodes), 256, 0, st>>>(A.nodes, A, kcut, s.status);
    GEV_TRY(last_error());
    if (top) {
      GEV_COUNT(s);
      k_count_out<<<nnodes, 32, 0, st>>>(A.nodes, A, kcut);
      GEV_CUDA_TRY(cudaMemcpyAsync(hn.data(), A.nodes, sizeof(Node) * nnodes, cudaMemcpyDeviceToHost, st));
      GEV_CUDA_TRY(cudaStreamSynchronize(st));
      top_deflated = hn[0].ndefl;
    }
    int Koutmax = 0;
    for (auto& x : hn) Koutmax = std::max(Koutmax, x.Kout);
    if (Koutmax > 0) {
      GEV_COUNT(s);
      k_vectors<<<dim3(Koutmax, nnodes), 256, 0, st>>>(A.nodes, A, U, ldq);
    }
    if (Tmax > 0) {
      GEV_COUNT(s);
      k_gather<<<dim3(Tmax, nnodes), 256, 0, st>>>(A.nodes, A, Qa, ldq, Qg, Qb);
    }
    GEV_TRY(last_error());
    // eigenvector update: top rows use the top-only and mixed columns, bottom rows the mixed and
    // bottom-only ones
    for (auto& x : hn) {
      if (x.Kout == 0) continue;
      const int n1 = x.m - x.a, n2 = x.c - x.m;
      const double* Ub = U + (long long)x.a * ldq;  // column a, rows 0 .. K-1 (gather order)
      if (x.K1 + x.K2 > 0)
      {
        GemmP<double> g = gp<double>(n1, x.Kout, x.K1 + x.K2, 0, 0, 1.0, Qg + x.a + (long long)x.a * ldq, ldq,
                                     Ub, ldq, 0.0, Qb + x.a + (long long)x.a * ldq, ldq);
        g.lowp = s.dc_lowp;
        gemm(s, g);
      }
      else
        GEV_CUDA_TRY(cudaMemset2DAsync(Qb + x.a + (long long)x.a * ldq, ldq * 8, 0, n1 * 8, x.Kout, st));
      if (x.K2 + x.K3 > 0)
      {
        GemmP<double> g = gp<double>(n2, x.Kout, x.K2 + x.K3, 0, 0, 1.0, Qg + x.m + (long long)(x.a + x.K1) * ldq,
                                     ldq, Ub + x.K1, ldq, 0.0, Qb + x.m + (long long)x.a * ldq, ldq);
        g.lowp = s.dc_lowp;
        gemm(s, g);
      }
      else
        GEV_CUDA_TRY(cudaMemset2DAsync(Qb + x.m + (long long)x.a * ldq, ldq * 8, 0, n2 * 8, x.Kout, st));
    }
    GEV_COUNT(s);
    k_finalize<<<dim3(cdiv(Tmax, 256), nnodes), 256, 0, st>>>(A.nodes, A, w);
    GEV_TRY(last_error());
    GEV_COUNT(s);
    k_copy_int<<<eb, 256, 0, st>>>(n, A.colmap2, A.colmap);
    std::swap(Qa, Qb);
  }
  // the k lowest eigenvectors
  GEV_COUNT(s);
  k_output<<<k, 256, 0, st>>>(n, k, Qa, ldq, A.colmap, Z, ldz);
  GEV_TRY(last_error());
  GEV_CUDA_TRY(cudaMemsetAsync(&s.status[ST_DEFLATED], 0, sizeof(int), st));
  GEV_CUDA_TRY(cudaMemcpyAsync(&s.status[ST_DEFLATED], &top_deflated, sizeof(int), cudaMemcpyHostToDevice, st));
  GEV_CUDA_TRY(cudaStreamSynchronize(st));
  if (deflated) *deflated = top_deflated;
  return 0;
}

}  // namespace gev
