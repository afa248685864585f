// Stage 2 of the two-stage tridiagonalisation: band (width b) -> real symmetric tridiagonal by
// bulge chasing, B = Q2 T' Q2^H, and the back-transform Y = Q2 D Z (D: diagonal phases that make
// the complex off-diagonal real).
//
// Sweep s (s = 0 .. n-3) annihilates column s below the subdiagonal with a Householder reflector
// H(s,0) on rows W_0 = [s+1, s+1+b); applying it two-sided fills the b x b block below the window
// (the bulge).  Task t >= 1 annihilates the first column of that block with H(s,t) on rows
// W_t = [s+1+tb, s+1+(t+1)b), and so on down the band.  Footprint of task (s,t): rows
// [p_t, p_{t+2}), columns [p_{t-1}, p_{t+1}) (p_t = s+1+tb).  Task (s+1,t) overlaps tasks
// (s,t-1) .. (s,t+2) only, so sweep s+1 may run task t once sweep s has finished task t+2.
//
// GPU mapping: one persistent cooperative kernel; block q owns sweeps q, q+G, q+2G, ... and runs
// their tasks in order, staging the three blocks of a task (L = (W_t, W_{t-1}), D = (W_t, W_t),
// E = (W_{t+1}, W_t)) in shared memory; E stays resident as the next task's L.  A per-sweep
// progress counter (release: __threadfence + store; acquire: volatile load + __threadfence, band
// reads through L2 with __ldcg) orders the sweeps.  Every wait is bounded (status[ST_SPIN] iterations
// when the host set a limit, else kSpinLimit, ~2 s): on expiry the kernel records ST_TIMEOUT, raises
// the abort flag and all blocks return.
//
// The band is stored compactly: element (i, j), 0 <= i-j < 2b, at band[(i-j) + j*ldb], ldb = 2b
// (rows b+1 .. 2b-1 below the diagonal hold the bulge).
#include <algorithm>
#include <climits>

#include <type_traits>

#include "common.cuh"
#include "coop.cuh"

namespace gev {

namespace {

constexpr int NT = 256;


__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ zd warp_sum(zd v) { return make_zd(warp_sum(v.x), warp_sum(v.y)); }
__device__ __forceinline__ float warp_sum(float v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ zf warp_sum(zf v) { return make_zf(warp_sum(v.x), warp_sum(v.y)); }

// Bounded acquire-wait until *flag >= target.  Thread 0 spins; returns false on timeout/abort.
__device__ bool wait_ge(const int* flag, int target, int* status, int* abort_flag, int site) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    int good = 1;
    volatile const int* vf = flag;
    volatile int* va = abort_flag;
    const long long lim = spin_limit(status);
    long long it = 0;
    while (*vf < target) {
      if (*va) { good = 0; break; }
      if (++it > lim) {
        atomicCAS(&status[ST_TIMEOUT], 0, site);
        atomicExch(abort_flag, 1);
        good = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// Band -> tridiagonal by bulge chasing (one sweep per block at a time).  Task t of sweep s
// annihilates the column below the band with one Householder reflector H = I - tau v v^H
// (v_0 = 1) acting on rows p .. p+len-1, p = s + 1 + t b:
//   L (the block left of the reflector's rows, the previous task's bulge) <- H L   (t > 0),
//   D (the diagonal block)                                                  <- H D H^H,
//   E (the block below D: the new bulge)                                    <- E H^H,
// and the reflector is kept for back-transform 2.  Sweep s+1 may run task t once sweep s has
// finished task t+2 (their blocks overlap up to there): a bounded wait on progress[s].
// A task is a short dependent chain, and on GB300 the FP64 pipe executes a warp-wide FP64
// instruction in ~19 cycles, so the FP64 form is bound by its count of FP64 instructions and the
// FP32 form by latency.  Hence: all arithmetic in the data's own precision R (FP32 for the mixed
// form); matrix-vector products with four threads per row / column (partial sums over every
// fourth term, combined through shared memory: all eight warps, hence all four schedulers' FP64
// pipes, take an equal share and no shuffle reductions are needed); element updates spread over
// all threads; the
// loads of the D and E blocks issued into registers right after the wait, so that their L2 latency
// overlaps the reflector and the update of L.
template <class T>
__global__ void __launch_bounds__(NT) k_bulge(int n, int b, T* band, int ldb, T* V2, T* tau2, int ntask,
                                              int* progress, int* status, int* abort_flag, int stall) {
  using R = typename real_of<T>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int PF = 64 * 64 / NT;  // register prefetch slots per thread (b <= 64)
  const int LD = b + 1;
  T* Ls = reinterpret_cast<T*>(smraw);
  T* Es = Ls + b * LD;
  T* Ds = Es + b * LD;
  T* v = Ds + b * LD;
  T* y = v + b;
  T* w = y + b;
  T* part4 = w + b;  // 4 x 64 partial sums of the matrix-vector products
  __shared__ T sh_tau, sh_beta, sh_scale;
  __shared__ R sh_c;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lb = __ffs(b) - 1;  // b is a power of two (16, 32, 64)
  const int ci = tid & (b - 1), cj = tid >> lb, cstep = NT >> lb;
  const int qi = tid & 63, qp = tid >> 6;  // matrix-vector products: row / column qi, quarter qp
  static_assert(NT == 256, "the products use 4 x 64 threads");

  for (int s = blockIdx.x; s <= n - 3; s += gridDim.x) {
    bool pendingL = false;
    for (int t = 0;; ++t) {
      const int p = s + 1 + t * b;
      const int len = (p < n) ? min(b, n - p) : 0;
      const int pp = p - b;
      // (stall: a failure-path test makes the first wait target a flag that nothing sets)
      if (s > 0 && !(stall ? wait_ge(&status[ST_STALL], 1, status, abort_flag, 202)
                           : wait_ge(&progress[s - 1], t + 3, status, abort_flag, 201)))
        return;
      if (t > 0 && len <= 1) {
        if (pendingL && len == 1)
          for (int q = tid; q < b; q += NT) stcg_(&band[(b - q) + (long long)(pp + q) * ldb], Ls[q * LD]);
        break;
      }
      const int p2 = p + len;
      const int len2 = (p2 < n) ? min(b, n - p2) : 0;
      // ---- prefetch D (lower triangle) and E into registers: thread (ci, cj) holds row ci,
      // columns cj, cj + cstep, ... of each block
      T dreg[PF], ereg[PF];
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int jj = cj + u * cstep;
        dreg[u] = (jj < len && ci < len && ci >= jj) ? ldcg_(&band[(ci - jj) + (long long)(p + jj) * ldb])
                                                     : zero_<T>();
        ereg[u] = (jj < len && ci < len2) ? ldcg_(&band[(len + ci - jj) + (long long)(p + jj) * ldb]) : zero_<T>();
      }
      // ---- generating vector x and the reflector
      for (int i = tid; i < len; i += NT)
        v[i] = (t == 0) ? ldcg_(&band[(1 + i) + (long long)s * ldb]) : Ls[i];
      __syncthreads();
      if (warp == 0) {
        R xn = 0;
        for (int i = 1 + lane; i < len; i += 32) xn += (R)abs2_(v[i]);
        xn = warp_sum(xn);
        if (lane == 0) {
          const T alpha = v[0];
          if (xn == (R)0 && im_(alpha) == 0) {
            sh_tau = zero_<T>();
            sh_beta = alpha;
            sh_scale = zero_<T>();
          } else {
            const R nrm = sqrt((R)abs2_(alpha) + xn);
            const T bt = from_re<T>(re_(alpha) >= 0 ? -nrm : nrm);
            sh_tau = div_(bt - alpha, bt);
            sh_beta = bt;
            sh_scale = div_(from_re<T>(1.0), alpha - bt);
          }
        }
      }
      __syncthreads();
      const T tau = sh_tau, beta = sh_beta, scale = sh_scale;
      for (int i = tid; i < len; i += NT) v[i] = (i == 0) ? from_re<T>(1.0) : scale * v[i];
      __syncthreads();
      // ---- (i) the annihilated column, (ii) left update of the rest of L, store L
      if (t == 0) {
        for (int i = tid; i < len; i += NT)
          stcg_(&band[(1 + i) + (long long)s * ldb], i == 0 ? beta : zero_<T>());
      } else {
        if (qi >= 1 && qi < b) {  // w_q = conj(tau) v^H L(:, q): four partial sums per column
          T acc = zero_<T>();
          for (int i = qp; i < len; i += 4) acc += cmul(v[i], Ls[i + qi * LD]);
          part4[qp * 64 + qi] = acc;
        }
        __syncthreads();
        if (tid >= 1 && tid < b)
          w[tid] = conj_(tau) * ((part4[tid] + part4[64 + tid]) + (part4[128 + tid] + part4[192 + tid]));
        __syncthreads();
        if (ci < len) {
          for (int q = (cj == 0 ? cstep : cj); q < b; q += cstep) Ls[ci + q * LD] -= v[ci] * w[q];
          if (cj == 0) Ls[ci] = (ci == 0) ? beta : zero_<T>();
        }
        __syncthreads();
        if (ci < len)
          for (int q = cj; q < b; q += cstep) stcg_(&band[(b + ci - q) + (long long)(pp + q) * ldb], Ls[ci + q * LD]);
      }
      // ---- (iii) two-sided update of the diagonal block
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int jj = cj + u * cstep;
        if (jj < len && ci < len && ci >= jj) {
          T val = dreg[u];
          if (ci == jj) val = from_re<T>(re_(val));
          Ds[ci + jj * LD] = val;
          Ds[jj + ci * LD] = conj_(val);
        }
        if (jj < len && ci < len2) Es[ci + jj * LD] = ereg[u];
      }
      __syncthreads();
      if (qi < len) {  // y = D v: four partial sums per row
        T acc = zero_<T>();
        for (int j = qp; j < len; j += 4) acc += Ds[qi + j * LD] * v[j];
        part4[qp * 64 + qi] = acc;
      }
      __syncthreads();
      if (tid < len) y[tid] = (part4[tid] + part4[64 + tid]) + (part4[128 + tid] + part4[192 + tid]);
      __syncthreads();
      if (warp == 0) {
        T acc = zero_<T>();
        for (int i = lane; i < len; i += 32) acc += cmul(v[i], y[i]);
        acc = warp_sum(acc);
        if (lane == 0) sh_c = (R)0.5 * (R)abs2_(tau) * (R)re_(acc);
      }
      __syncthreads();
      for (int i = tid; i < len; i += NT) y[i] = tau * y[i] - from_re<T>(sh_c) * v[i];
      __syncthreads();
      if (ci < len)
        for (int jj = cj; jj <= ci; jj += cstep) {
          T val = Ds[ci + jj * LD] - (mulc(y[ci], v[jj]) + mulc(v[ci], y[jj]));
          if (ci == jj) val = from_re<T>(re_(val));
          stcg_(&band[(ci - jj) + (long long)(p + jj) * ldb], val);
        }
      // ---- (iv) right update of the block below: creates the next bulge
      if (len2 > 0) {
        if (qi < len2) {  // w = tau E v: four partial sums per row
          T acc = zero_<T>();
          for (int q = qp; q < len; q += 4) acc += Es[qi + q * LD] * v[q];
          part4[qp * 64 + qi] = acc;
        }
        __syncthreads();
        if (tid < len2) w[tid] = tau * ((part4[tid] + part4[64 + tid]) + (part4[128 + tid] + part4[192 + tid]));
        __syncthreads();
        if (ci < len2)
          for (int q = cj; q < len; q += cstep) Es[ci + q * LD] -= mulc(w[ci], v[q]);
        pendingL = true;
      } else {
        pendingL = false;
      }
      // ---- keep the reflector for the back-transform
      const long long rid = (long long)s * ntask + t;
      for (int i = tid; i < b; i += NT) V2[rid * b + i] = (i < len) ? v[i] : zero_<T>();
      if (tid == 0) tau2[rid] = tau;
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        atomicExch(&progress[s], t + 1);
      }
      T* tmp = Ls;
      Ls = Es;
      Es = tmp;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicExch(&progress[s], INT_MAX);
    }
  }
}

// d = Re diag, e = |subdiag| with the phase recursion phi_0 = 1, phi_{i+1} = phi_i eps_i/|eps_i|
// (complex), or e = subdiag (real).  One block: the phase recursion is sequential.
template <class T>
// (the phases are formed in FP64 also from an FP32 band, so that their product over n steps stays
// accurate)
__global__ void k_tridiag_out(int n, const T* band, int ldb, double* d, double* e, zd* phase) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = re_(band[(long long)i * ldb]);
  if constexpr (is_cx<T>::value) {
    if (threadIdx.x == 0) {
      zd ph = make_zd(1.0, 0.0);
      phase[0] = ph;
      for (int i = 0; i + 1 < n; ++i) {
        const T eps = band[1 + (long long)i * ldb];
        const double ex = re_(eps), ey = im_(eps);
        const double a = hypot(ex, ey);
        e[i] = a;
        if (a > 0.0) ph = ph * make_zd(ex / a, ey / a);
        phase[i + 1] = ph;
      }
    }
  } else {
    for (int i = threadIdx.x; i + 1 < n; i += blockDim.x) e[i] = band[1 + (long long)i * ldb];
  }
}

// Y = D Z (real Z -> scalar type; D = diag(phase) for complex data, identity for real).
template <class T>
__global__ void k_phase_rows(int n, int k, const double* Z, long long ldz, const zd* phase, T* Y,
                             long long ldy) {
  const long long total = (long long)n * k;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), c = (int)(t / n);
    const double z = Z[i + c * ldz];
    if constexpr (is_cx<T>::value) {
      const zd v = z * phase[i];
      Y[i + c * ldy] = T{(decltype(T{}.x))v.x, (decltype(T{}.x))v.y};
    } else {
      Y[i + c * ldy] = (T)z;
    }
  }
}

// Y <- Q2 Y, level-parallel.  With G = b sweeps per group, the block D_t^g of group g
// (reflectors H(s, t), s = gb .. gb+b-1, applied in the order s descending) acts on the row window
// [(g+t) b + 1, (g+t+2) b - 1).  Q2 = P_0 P_1 ... with P_g = D_T^g ... D_1^g D_0^g, so Y <- Q2 Y
// applies D_0^last first.  D_t^g must follow D_{t-1}^g and D_{t'}^{g+1} for t' <= t (overlapping
// windows), which is exactly the order of the levels L = t + (ngroups - 1 - g); blocks of one level
// have windows 2b apart, act on disjoint rows and commute.  One launch per level: blockIdx.x picks
// the group, blockIdx.y a block of columns of Y, one thread per column (all FMAs of a thread are
// on its own column; the reflector entries are shared-memory broadcasts).
template <class T, int COLS>
__global__ void __launch_bounds__(COLS) k_bt_bulge_level(int n, int k, int b, int L, int ngroups,
                                                         const T* V2, const T* tau2, int ntask, T* Y,
                                                         long long ldy) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = max(0, ngroups - 1 - L) + blockIdx.x;
  const int t = L - (ngroups - 1 - g);
  if (g >= ngroups || t < 0 || t >= ntask) return;
  const int G = b;
  const int s0 = g * G;
  const int last_sweep = n - 3;
  const int s1 = min(s0 + G - 1, last_sweep);
  const int w0 = s0 + 1 + t * b;
  if (w0 >= n) return;
  const int w1 = min(n, s1 + 1 + t * b + b);
  const int rows = w1 - w0;
  const int c = blockIdx.y * COLS + threadIdx.x;
  T* Zw = reinterpret_cast<T*>(smraw);   // rows x COLS (row-major)
  T* Vs = Zw + (size_t)(2 * b) * COLS;   // G x b
  T* ts = Vs + (size_t)G * b;            // G
  const int ncols = min(COLS, k - (int)blockIdx.y * COLS);
  for (int idx = threadIdx.x; idx < (s1 - s0 + 1) * b; idx += COLS) {
    const int q = idx / b, i = idx % b;
    Vs[q * b + i] = V2[((long long)(s0 + q) * ntask + t) * b + i];
  }
  for (int q = threadIdx.x; q <= s1 - s0; q += COLS) ts[q] = tau2[(long long)(s0 + q) * ntask + t];
  if (threadIdx.x < ncols)
    for (int r = 0; r < rows; ++r) Zw[r * COLS + threadIdx.x] = Y[(w0 + r) + (long long)c * ldy];
  __syncthreads();
  if (threadIdx.x < ncols) {
    for (int q = s1 - s0; q >= 0; --q) {
      const T tau = ts[q];
      if (tau == zero_<T>()) continue;
      const int p = s0 + q + 1 + t * b;
      const int len = min(b, n - p);
      const int off = p - w0;
      const T* vq = Vs + q * b;
      T acc = zero_<T>();
      for (int i = 0; i < len; ++i) acc += cmul(vq[i], Zw[(off + i) * COLS + threadIdx.x]);
      acc = tau * acc;
      for (int i = 0; i < len; ++i) Zw[(off + i) * COLS + threadIdx.x] -= vq[i] * acc;
    }
    for (int r = 0; r < rows; ++r) Y[(w0 + r) + (long long)c * ldy] = Zw[r * COLS + threadIdx.x];
  }
}

// FP32 form of the level kernel: the same (group, task) blocks and level order, but each thread
// applies the reflectors to its column from registers.  The 64 reflectors of a block are taken in
// chunks of 8 (descending): a chunk touches window rows [q0, q0 + B + 7), which are moved from the
// staged shared-memory window into registers, updated by the 8 reflectors (dot products with four
// partial sums) and written back.  Reflector entries are shared-memory broadcasts, zero-padded
// beyond the matrix end, so every chunk runs the same straight-line code.
constexpr int BTF_COLS = 128, BTF_CH = 8;
template <int B>
__global__ void __launch_bounds__(BTF_COLS) k_bt_level_f32(int n, int k, int L, int ngroups, const float* V2,
                                                           const float* tau2, int ntask, float* Y, long long ldy) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = max(0, ngroups - 1 - L) + blockIdx.x;
  const int t = L - (ngroups - 1 - g);
  if (g >= ngroups || t < 0 || t >= ntask) return;
  const int s0 = g * B;
  const int s1 = min(s0 + B - 1, n - 3);
  const int w0 = s0 + 1 + t * B;
  if (w0 >= n) return;
  const int rows = min(n, s1 + 1 + t * B + B) - w0;  // <= 2B - 1
  constexpr int LDZ = BTF_COLS + 1;
  float* Zs = reinterpret_cast<float*>(smraw);          // 2B x LDZ
  float* Vs = Zs + 2 * B * LDZ;                          // B x B (16-byte aligned rows)
  float* ts = Vs + B * B;                                // B
  const int c0 = blockIdx.y * BTF_COLS;
  const int ncols = min(BTF_COLS, k - c0);
  for (int idx = threadIdx.x; idx < B * B; idx += BTF_COLS) {
    const int q = idx / B, i = idx % B;
    const int p = s0 + q + 1 + t * B;
    float v = 0.f;
    if (s0 + q <= s1 && i < n - p) v = V2[((long long)(s0 + q) * ntask + t) * B + i];
    Vs[idx] = v;
  }
  for (int q = threadIdx.x; q < B; q += BTF_COLS) ts[q] = (s0 + q <= s1) ? tau2[(long long)(s0 + q) * ntask + t] : 0.f;
  for (int idx = threadIdx.x; idx < 2 * B * BTF_COLS; idx += BTF_COLS) {
    const int r = idx % (2 * B), c = idx / (2 * B);  // consecutive threads: consecutive rows
    float v = 0.f;
    if (r < rows && c < ncols) v = Y[(w0 + r) + (long long)(c0 + c) * ldy];
    Zs[r * LDZ + c] = v;
  }
  __syncthreads();
  const int c = threadIdx.x;
  for (int q0 = B - BTF_CH; q0 >= 0; q0 -= BTF_CH) {
    float z[B + BTF_CH - 1];
#pragma unroll
    for (int j = 0; j < B + BTF_CH - 1; ++j) z[j] = Zs[(q0 + j) * LDZ + c];
#pragma unroll
    for (int u = BTF_CH - 1; u >= 0; --u) {
      const float4* v4 = reinterpret_cast<const float4*>(Vs + (q0 + u) * B);
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
      for (int i = 0; i < B / 4; ++i) {
        const float4 v = v4[i];
        a0 = fmaf(v.x, z[u + 4 * i], a0);
        a1 = fmaf(v.y, z[u + 4 * i + 1], a1);
        a2 = fmaf(v.z, z[u + 4 * i + 2], a2);
        a3 = fmaf(v.w, z[u + 4 * i + 3], a3);
      }
      const float w = ts[q0 + u] * ((a0 + a1) + (a2 + a3));
#pragma unroll
      for (int i = 0; i < B / 4; ++i) {
        const float4 v = v4[i];
        z[u + 4 * i] = fmaf(-v.x, w, z[u + 4 * i]);
        z[u + 4 * i + 1] = fmaf(-v.y, w, z[u + 4 * i + 1]);
        z[u + 4 * i + 2] = fmaf(-v.z, w, z[u + 4 * i + 2]);
        z[u + 4 * i + 3] = fmaf(-v.w, w, z[u + 4 * i + 3]);
      }
    }
#pragma unroll
    for (int j = 0; j < B + BTF_CH - 1; ++j) Zs[(q0 + j) * LDZ + c] = z[j];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 2 * B * BTF_COLS; idx += BTF_COLS) {
    const int r = idx % (2 * B), cc = idx / (2 * B);
    if (r < rows && cc < ncols) Y[(w0 + r) + (long long)(c0 + cc) * ldy] = Zs[r * LDZ + cc];
  }
}

// Compact-WY form of one level's reflector blocks, for the tensor-core back-transform: for block j
// (group g = g_lo + j, task t) with reflectors v_q = V(:, q) of sweeps s0 + q on the window rows
// [w0, w0 + 2b) (v_q non-zero in rows q .. q + b - 1, v_q(q) = 1),
//   D_j = H(s0) H(s0 + 1) ... H(s0 + b - 1) = I - V T V^H,  T upper triangular:
//   T_qq = tau_q,  T(0:q, q) = -tau_q T(0:q, 0:q) (V(:, 0:q)^H v_q),
// and W_j = V T (2b x b, column-major at W + j 2b b) is written for the second product.  A reflector
// with tau = 0 (a task that never ran) is a zero column.  One block of 256 threads per D_j: the Gram
// entries V^H V by all threads (padded shared-memory columns), the recurrence by one warp, W by all.
// The blocks of level L: groups g in [g_lo, g_lo + nblk) with task t = L - (ngroups - 1 - g) in
// range and a window start w0(g) = (2g + L - ngroups + 1) b + 1 below n; w00 = w0(g_lo); windows are
// 2b apart.  (Host and device.)
struct LevelBlocks {
  int g_lo, nblk, w00;
};
__host__ __device__ inline LevelBlocks level_blocks(int n, int b, int L, int ngroups, int ntask) {
  LevelBlocks lb{0, 0, 0};
  const int g_lo = max(0, ngroups - 1 - L);
  int g_hi = min(ngroups - 1, ntask - 1 + ngroups - 1 - L);
  while (g_hi >= g_lo && (2 * g_hi + L - ngroups + 1) * b + 1 >= n) --g_hi;
  if (g_hi < g_lo) return lb;
  lb.g_lo = g_lo;
  lb.nblk = g_hi - g_lo + 1;
  lb.w00 = (2 * g_lo + L - ngroups + 1) * b + 1;
  return lb;
}

// Levels L0 .. L0 + nL - 1 in one grid: block x is block j of level L (levels in order), and its W
// goes to W + (blocks of the earlier levels of the range + j) 2b b.
template <class T>
__global__ void __launch_bounds__(256) k_wy_level(int n, int b, int L0, int nL, int ngroups, int ntask,
                                                  const T* V2, const T* tau2, T* W) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tid = threadIdx.x;
  int j = blockIdx.x, L = L0, before = 0;
  LevelBlocks lb = level_blocks(n, b, L, ngroups, ntask);
  while (j >= lb.nblk && L < L0 + nL - 1) {
    j -= lb.nblk;
    before += lb.nblk;
    ++L;
    lb = level_blocks(n, b, L, ngroups, ntask);
  }
  if (j >= lb.nblk) return;
  const int g_lo = lb.g_lo, w00 = lb.w00;
  W += (size_t)before * 2 * b * b;
  const int g = g_lo + j, t = L - (ngroups - 1 - g);
  const int m = 2 * b, ldv = m + 1;     // padded: column q of V starts q (2b + 1) elements in
  T* Vs = reinterpret_cast<T*>(smraw);  // 2b x b (ld 2b + 1)
  T* Gs = Vs + (size_t)ldv * b;         // b x b Gram V^H V, then overwritten by T (strict upper part)
  T* taus = Gs + (size_t)b * (b + 1);   // b
  const int ldg = b + 1;
  const int w0 = w00 + m * j;
  for (int idx = tid; idx < m * b; idx += blockDim.x) {
    const int r = idx % m, q = idx / m;
    const int sw = g * b + q, rel = r - q;
    T v = zero_<T>();
    if (sw <= n - 3 && rel >= 0 && rel < b && w0 + r < n) {
      const long long rid = (long long)sw * ntask + t;
      if (tau2[rid] != zero_<T>()) v = V2[rid * b + rel];
    }
    Vs[r + q * ldv] = v;
  }
  for (int q = tid; q < b; q += blockDim.x) {
    const int sw = g * b + q;
    taus[q] = (sw <= n - 3) ? tau2[(long long)sw * ntask + t] : zero_<T>();
  }
  __syncthreads();
  // Gram entries G(p, q) = v_p^H v_q, p < q (rows q .. p + b - 1 overlap)
  for (int idx = tid; idx < b * b; idx += blockDim.x) {
    const int p = idx % b, q = idx / b;
    if (p < q) {
      T acc = zero_<T>();
      for (int r = q; r < p + b; ++r) acc += cmul(Vs[r + p * ldv], Vs[r + q * ldv]);
      Gs[p + q * ldg] = acc;
    }
  }
  __syncthreads();
  // T by columns, in place over the Gram matrix's strict upper part: column q needs G(0:q, q) and the
  // finished columns 0 .. q-1 of T (diagonal: tau); one warp, two entries per lane (b <= 64)
  if (tid < 32) {
    for (int q = 0; q < b; ++q) {
      const T tq = taus[q];
      T out[2];
      for (int h = 0; h < 2; ++h) {
        const int p = tid + 32 * h;
        out[h] = zero_<T>();
        if (p < q) {
          T acc = zero_<T>();
          for (int l = p; l < q; ++l) acc += ((l == p) ? taus[p] : Gs[p + l * ldg]) * Gs[l + q * ldg];
          out[h] = -(tq * acc);
        }
      }
      __syncwarp();
      for (int h = 0; h < 2; ++h) {
        const int p = tid + 32 * h;
        if (p < q) Gs[p + q * ldg] = out[h];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // W = V T: W(r, q) = sum_{p <= q} V(r, p) T(p, q), V(r, p) != 0 for r - b < p <= r (T_pp = tau_p)
  T* Wj = W + (size_t)j * m * b;
  for (int idx = tid; idx < m * b; idx += blockDim.x) {
    const int r = idx % m, q = idx / m;
    const int p0 = max(0, r - b + 1), p1 = min(q, r);
    T acc = zero_<T>();
    for (int p = p0; p <= p1; ++p) acc += Vs[r + p * ldv] * ((p == q) ? taus[q] : Gs[p + q * ldg]);
    Wj[idx] = acc;
  }
}

template <class T> size_t bulge_smem(int b) { return sizeof(T) * ((size_t)3 * b * (b + 1) + 3 * b + 4 * 64) + 64; }

}  // namespace

template <class T> int hb2st(Sys& s, double* d, double* e) {
  const int n = s.n, b = s.band_b_used;
  const int ldb = 2 * b;
  T* band = (T*)s.band;
  if (n <= 2) {
    // already tridiagonal
  } else {
    if (b > 64) return GEV_ERR_UNSUPPORTED;
    const size_t smem = bulge_smem<T>(b);
    GEV_TRY(allow_max_dyn_smem(k_bulge<T>));
    int per_sm = 0;
    GEV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bulge<T>, NT, smem));
    if (per_sm < 1) return GEV_ERR_UNSUPPORTED;
    // Sweep s+1 trails sweep s by three tasks and a sweep runs (n - s) / b tasks, so at most about
    // n / (3b) sweeps are in flight: more blocks would only hold SMs (in a spin wait) that other
    // streams' work - concurrent solves of the serving form - could use.
    int G = per_sm * s.sms;
    const int inflight = n / (3 * b) + 8;
    if (G > inflight) G = inflight;
    if (G > n - 2) G = n - 2;
    GEV_CUDA_TRY(cudaMemsetAsync(s.prog, 0, sizeof(int) * (size_t)n, s.stream));
    GEV_CUDA_TRY(cudaMemsetAsync(s.tau2, 0, s.es() * (size_t)n * s.ntask, s.stream));
    // The FP32 back-transform applies every stored slot with its tau (no branch), so the slots of
    // tasks that never ran (a sweep ends without storing a reflector for its last single row) must
    // hold zeros, not whatever the workspace held before: 0 * NaN would poison the column.
    if constexpr (std::is_same<T, float>::value)
      GEV_CUDA_TRY(cudaMemsetAsync(s.V2, 0, sizeof(T) * (size_t)b * n * s.ntask, s.stream));
    GEV_CUDA_TRY(cudaMemsetAsync(&s.status[ST_ABORT], 0, sizeof(int), s.stream));
    int nn = n, bb = b, lb = ldb, nt = s.ntask;
    T* V2 = (T*)s.V2;
    T* tau2 = (T*)s.tau2;
    int* prog = s.prog;
    int* st = s.status;
    int* ab = &s.status[ST_ABORT];
    int stall = s.opts.debug_stall ? 1 : 0;
    void* args[] = {&nn, &bb, &band, &lb, &V2, &tau2, &nt, &prog, &st, &ab, &stall};
    GEV_COUNT(s);
    GEV_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_bulge<T>, dim3(G), dim3(NT), args, smem, s.stream));
  }
  GEV_COUNT(s);
  k_tridiag_out<T><<<1, 256, 0, s.stream>>>(n, band, ldb, d, e, (zd*)s.phase);
  GEV_TRY(last_error());
  s.have_tridiag_refl = true;
  return 0;
}

template <class T, int COLS> int bt_levels(Sys& s, int n, int k, int b, T* Y, int ldy);


// Y <- Q2 Y with every level applied as  P = blockdiag(V_j^H) Y_L,  Y_L -= blockdiag(V_j T_j) P  on the
// emulated FP64 product engine (Y_L: the level's rows).  Returns GEV_ERR_UNSUPPORTED, before
// launching anything, when the handle's scratch cannot hold a level's product.
template <class T> int bt_levels_wy(Sys& s, int n, int k, int b, T* Y, int ldy) {
  constexpr int cx = is_cx<T>::value ? 1 : 0;
  constexpr bool f32 = std::is_same<T, float>::value;
  const int ngroups = (n - 3) / b + 1;
  const int nlevels = ngroups + s.ntask;
  T* P = (T*)s.W1;  // (nblk b) x k products V^H Y (W1 is free during the back-transform)
  T* Wb = (T*)s.Q;  // the W_j blocks of LCHUNK consecutive levels (Q is free once the divide and conquer is done)
  constexpr int LCHUNK = 16;
  size_t need = 0;
  int max_nblk = 0;
  for (int L = 0; L < nlevels; ++L) {
    const LevelBlocks lb = level_blocks(n, b, L, ngroups, s.ntask);
    if (lb.nblk == 0) continue;
    max_nblk = std::max(max_nblk, lb.nblk);
    const int rows = std::min(lb.nblk * 2 * b, n - lb.w00);
    if constexpr (f32) {
      need = std::max(need, gemm_f32_bdiag_scratch(lb.nblk * b, k, rows, b, 2 * b));
      need = std::max(need, gemm_f32_bdiag_scratch(rows, k, lb.nblk * b, 2 * b, b));
    } else {
      need = std::max(need, gemm_f64_bdiag_scratch(lb.nblk * b, k, rows, b, 2 * b, cx));
      need = std::max(need, gemm_f64_bdiag_scratch(rows, k, lb.nblk * b, 2 * b, b, cx));
    }
  }
  if (need > s.ozws_bytes || (size_t)max_nblk * b * k * sizeof(T) > (size_t)n * n * sizeof(T) ||
      (size_t)LCHUNK * max_nblk * 2 * b * b * sizeof(T) > (size_t)n * n * sizeof(double))
    return GEV_ERR_UNSUPPORTED;
  const size_t smem = sizeof(T) * ((size_t)(2 * b + 1) * b + (size_t)b * (b + 1) + b) + 64;
  GEV_TRY(allow_dyn_smem(k_wy_level<T>, smem));
  size_t woff = 0;  // offset of level L's blocks in Wb (elements)
  for (int L = 0; L < nlevels; ++L) {
    if (L % LCHUNK == 0) {  // the compact-WY blocks of the next LCHUNK levels, in one grid
      int nb = 0;
      for (int l = L; l < std::min(nlevels, L + LCHUNK); ++l) nb += level_blocks(n, b, l, ngroups, s.ntask).nblk;
      if (nb > 0) {
        GEV_COUNT(s);
        k_wy_level<T><<<nb, 256, smem, s.stream>>>(n, b, L, std::min(LCHUNK, nlevels - L), ngroups, s.ntask,
                                                   (const T*)s.V2, (const T*)s.tau2, Wb);
      }
      woff = 0;
    }
    const LevelBlocks lb = level_blocks(n, b, L, ngroups, s.ntask);
    if (lb.nblk == 0) continue;
    const int rows = std::min(lb.nblk * 2 * b, n - lb.w00);
    T* Wl = Wb + woff;
    woff += (size_t)lb.nblk * 2 * b * b;
    BdOp a1{1, cx, b, n, s.ntask, lb.g_lo, L, ngroups, lb.nblk, lb.w00, s.V2, s.tau2, nullptr};
    T* Yl = Y + lb.w00;
    const int M1 = lb.nblk * b;
    BdOp a2{2, cx, b, n, s.ntask, lb.g_lo, L, ngroups, lb.nblk, lb.w00, nullptr, nullptr, Wl};
    if constexpr (f32) {
      if (!gemm_f32_bdiag(s, M1, k, rows, a1, b, 2 * b, Yl, ldy, 1.f, 0.f, P, M1)) return GEV_ERR_CUDA;
      if (!gemm_f32_bdiag(s, rows, k, M1, a2, 2 * b, b, P, M1, -1.f, 1.f, Yl, ldy)) return GEV_ERR_CUDA;
    } else {
      // From orthonormal Z (s.z_unit), Y's columns stay unit vectors under the orthogonal transforms
      // (|y_ij| <= 1), and |P_qj| = |v_q^H y_j| <= ||v_q|| <= sqrt(2) (a Householder vector with
      // v(0) = 1): both below 2, so their scales need no pass over the data
      const bool u = s.z_unit;
      if (!gemm_f64_bdiag(s, M1, k, rows, a1, b, 2 * b, Yl, ldy, 1.0, 0.0, P, M1, u)) return GEV_ERR_CUDA;
      if (!gemm_f64_bdiag(s, rows, k, M1, a2, 2 * b, b, P, M1, -1.0, 1.0, Yl, ldy, u)) return GEV_ERR_CUDA;
    }
  }
  return last_error();
}

template <int B> int bt_levels_f32(Sys& s, int n, int k, float* Y, int ldy) {
  const int ngroups = (n - 3) / B + 1;
  const size_t smem = sizeof(float) * ((size_t)2 * B * (BTF_COLS + 1) + (size_t)B * B + B) + 64;
  GEV_TRY(allow_max_dyn_smem(k_bt_level_f32<B>));
  const int nlevels = ngroups + s.ntask;
  const unsigned ycb = cdiv(k, BTF_COLS);
  for (int L = 0; L < nlevels; ++L) {
    const int gmin = ngroups - 1 - L > 0 ? ngroups - 1 - L : 0;
    GEV_COUNT(s);
    k_bt_level_f32<B><<<dim3(ngroups - gmin, ycb), BTF_COLS, smem, s.stream>>>(
        n, k, L, ngroups, (const float*)s.V2, (const float*)s.tau2, s.ntask, Y, ldy);
  }
  return last_error();
}

// Y (n x k) = Q2 D Z for real Z.
template <class T> int bt_hb2st(Sys& s, const double* Z, int ldz, int k, T* Y, int ldy) {
  const int n = s.n, b = s.band_b_used;
  {
    long long total = (long long)n * k;
    unsigned blocks = cdiv(total, 256);
    if (blocks > 16u * s.sms) blocks = 16u * s.sms;
    GEV_COUNT(s);
    k_phase_rows<T><<<blocks, 256, 0, s.stream>>>(n, k, Z, ldz, (const zd*)s.phase, Y, ldy);
    GEV_TRY(last_error());
  }
  if (n <= 2) return 0;
  if constexpr (std::is_same<T, float>::value) {
    // (the block-diagonal BF16x6 form, bt_levels_wy<float>, measured slower than this register kernel
    // at n = 16384: 747 ms against 556 ms, its split passes and short-K products being latency bound)
    if (b == 16) return bt_levels_f32<16>(s, n, k, Y, ldy);
    if (b == 32) return bt_levels_f32<32>(s, n, k, Y, ldy);
    if (b == 64) return bt_levels_f32<64>(s, n, k, Y, ldy);
  }
  // FP64 data with the emulated product engine: each level as two block-diagonal tensor-core
  // products of its compact-WY blocks
  if constexpr (std::is_same<T, double>::value || std::is_same<T, zd>::value) {
    if (s.emu_fp64) {
      const int r = bt_levels_wy<T>(s, n, k, b, Y, ldy);
      if (r != GEV_ERR_UNSUPPORTED) return r;  // else: the scratch is too small, take the level kernel
    }
  }
  // level-parallel application (see k_bt_bulge_level); one thread per column, as many columns
  // per block as the staged window (2b rows) allows in shared memory
  const size_t per_col = sizeof(T) * 2 * (size_t)b;
  if (per_col * 256 <= (size_t)160 * 1024) return bt_levels<T, 256>(s, n, k, b, Y, ldy);
  if (per_col * 128 <= (size_t)160 * 1024) return bt_levels<T, 128>(s, n, k, b, Y, ldy);
  return bt_levels<T, 64>(s, n, k, b, Y, ldy);
}

template <class T, int COLS> int bt_levels(Sys& s, int n, int k, int b, T* Y, int ldy) {
  const int G = b;
  const int last_sweep = n - 3;
  const int ngroups = last_sweep / G + 1;
  const size_t smem = sizeof(T) * ((size_t)2 * b * COLS + (size_t)G * b + G) + 64;
  GEV_TRY(allow_max_dyn_smem(k_bt_bulge_level<T, COLS>));
  const int nlevels = ngroups + s.ntask;
  const unsigned ycb = cdiv(k, COLS);
  for (int L = 0; L < nlevels; ++L) {
    const int gmin = ngroups - 1 - L > 0 ? ngroups - 1 - L : 0;
    const int nblk = ngroups - gmin;
    GEV_COUNT(s);
    k_bt_bulge_level<T, COLS><<<dim3(nblk, ycb), COLS, smem, s.stream>>>(
        n, k, b, L, ngroups, (const T*)s.V2, (const T*)s.tau2, s.ntask, Y, ldy);
  }
  return last_error();
}

template int hb2st<double>(Sys&, double*, double*);
template int hb2st<float>(Sys&, double*, double*);
template int bt_hb2st<float>(Sys&, const double*, int, int, float*, int);
template int hb2st<zd>(Sys&, double*, double*);
template int bt_hb2st<double>(Sys&, const double*, int, int, double*, int);
template int bt_hb2st<zd>(Sys&, const double*, int, int, zd*, int);
template int hb2st<zf>(Sys&, double*, double*);
template int bt_hb2st<zf>(Sys&, const double*, int, int, zf*, int);

}  // namespace gev
