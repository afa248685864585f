// Stage 1 of the two-stage tridiagonalisation ("ELPA2", section "Usability and Tutorials"):
// full Hermitian A -> band B of width b, A = Q1 B Q1^H, and the matching back-transform Y = Q1 Z.
//
// For each panel (columns j0..j0+b-1, rows r0 = j0+b .. n-1):
//   1. Householder QR of the m x b panel (m = n - r0) in ONE cooperative kernel: the panel rows are
//      spread over all SMs and stay in shared memory; each column needs two bounded grid barriers
//      (norm, then the reflector's inner products, which also give the column of the compact-WY
//      factor T).  Q = H_0 ... H_{b-1} = I - Y T Y^H, T upper triangular.
//   2. Two-sided update of the trailing block A22 <- Q^H A22 Q by GEMMs:
//        W = A22 Y T,  U = T^H (Y^H W),  V = W - Y U / 2,  A22 -= [Y V] [V Y]^H (lower, one
//        rank-2b product), mirror.
// Y is kept explicitly (unit diagonal, zeros above) in the handle's V1 at the panel's position and
// T in T1, for the back-transform  Y_out = Q1 Z = Q_0 (Q_1 (... Q_last Z)).
#include <algorithm>

#include "common.cuh"
#include "coop.cuh"

namespace gev {

namespace {

constexpr int NT = 256;

template <class T>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;  // valid in thread 0
}

// One grid barrier per column.  Before the barrier every block sums, over its rows below the pivot,
// ||x||^2, u_j = sum_r conj(x_r) P(r, j) (j > c, the columns to update) and t_j = sum_r conj(P(r, j)) x_r
// (j < c, the stored reflectors, for T), with the UNSCALED column x; the block holding the pivot row
// publishes that row.  After the barrier each block forms the reflector (beta, tau, scale: v_c = 1,
// v_r = scale x_r) and recovers the inner products exactly as
//   w_j = v^H P(:, j) = P(c, j) + conj(scale) u_j,     s_j = Y(:, j)^H v = conj(P(c, j)) + scale t_j.
// The partial-sum buffers alternate with the column's parity: a block may start column c + 1 while a
// slower one still reads column c's sums, but column c + 2 waits for everyone at barrier c + 1.
template <class T>
__global__ void __launch_bounds__(NT) k_panel_qr(int m, int b, T* P, long long ldp, T* Y, long long ldy,
                                                 T* Tm, double* nrm_part, T* w_part, T* prow,
                                                 GridBar gb, int R, int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int blk = blockIdx.x, tid = threadIdx.x;
  const int lo = blk * R;
  const int hi = min(m, lo + R);
  const int rows = max(0, hi - lo);
  const long long lds = R | 1;
  const int G = gridDim.x;
  T* sm = reinterpret_cast<T*>(smraw);
  T* scratch = use_smem ? sm + lds * b : sm;
  T* red2 = scratch;          // NT entries
  T* wv = scratch + NT;       // b entries
  double* red = reinterpret_cast<double*>(wv + b);  // 32 doubles
  __shared__ T sh_tau, sh_beta, sh_scale;
  __shared__ int sh_trivial;

  T* base = use_smem ? sm : P + lo;
  const long long ld = use_smem ? lds : ldp;
  if (use_smem) {
    for (int idx = tid; idx < rows * b; idx += NT) {
      int r = idx % rows, c = idx / rows;
      sm[r + c * lds] = P[(lo + r) + c * ldp];
    }
    __syncthreads();
  }
  const int NG = NT / b;  // row groups (b is a power of two <= 128)
  const int jj = tid % b, grp = tid / b;

  for (int c = 0; c < b; ++c) {
    if (c >= m) {
      if (blk == 0 && tid < b) Tm[tid + c * b] = zero_<T>();
      continue;
    }
    const int par = c & 1;
    double* np_ = nrm_part + (size_t)par * G;
    T* wp_ = w_part + (size_t)par * G * b;
    T* pr_ = prow + (size_t)par * b;
    // ---- A: partial sums over this block's rows strictly below the pivot, unscaled column x
    const int r0 = max(0, c + 1 - lo);
    double ss = 0.0;
    for (int r = r0 + tid; r < rows; r += NT) ss += abs2_(base[r + c * ld]);
    const double tot = block_sum<T>(ss, red);
    {
      T acc = zero_<T>();
      if (grp < NG && jj != c)
        for (int r = r0 + grp; r < rows; r += NG) {
          const T x = base[r + c * ld], pj = base[r + jj * ld];
          acc += (jj > c) ? cmul(x, pj) : cmul(pj, x);
        }
      red2[tid] = acc;
      __syncthreads();
      if (tid < b) {
        T sum = zero_<T>();
        for (int g = 0; g < NG; ++g) sum += red2[g * b + tid];
        wp_[(long long)blk * b + tid] = sum;
      }
    }
    if (tid == 0) np_[blk] = tot;
    if (lo <= c && c < hi && tid < b) pr_[tid] = base[(c - lo) + tid * ld];  // the pivot row
    if (!grid_sync(gb, 101)) return;
    // ---- B: the reflector (all blocks compute it from the same sums, in a fixed order)
    double xpart = 0.0;
    for (int q = tid; q < G; q += NT) xpart += ldcg_(&np_[q]);
    const double xn_all = block_sum<T>(xpart, red);
    if (tid == 0) {
      const double xn = xn_all;
      const T alpha = ldcg_(&pr_[c]);
      const int trivial = (xn == 0.0 && im_(alpha) == 0.0);
      if (trivial) {
        sh_tau = zero_<T>();
        sh_beta = alpha;
        sh_scale = zero_<T>();
      } else {
        const double nrm = sqrt(abs2_(alpha) + xn);
        const double beta = re_(alpha) >= 0.0 ? -nrm : nrm;
        const T bt = from_re<T>(beta);
        sh_tau = div_(bt - alpha, bt);
        sh_beta = bt;
        sh_scale = div_(from_re<T>(1.0), alpha - bt);
      }
      sh_trivial = trivial;
    }
    __syncthreads();
    const T tau = sh_tau;
    if (sh_trivial) {
      if (blk == 0 && tid < b) Tm[tid + c * b] = zero_<T>();
      continue;  // uniform over the grid: every block computed the same reflector
    }
    const T scale = sh_scale;
    // the block partials of u / t, summed by NG threads per column, then in a fixed order
    {
      T part = zero_<T>();
      if (grp < NG)
        for (int q = grp; q < G; q += NG) part += ldcg_(&wp_[(long long)q * b + jj]);
      red2[tid] = part;
      __syncthreads();
      if (tid < b) {
        T sum = zero_<T>();
        for (int g = 0; g < NG; ++g) sum += red2[g * b + tid];
        const T pc = ldcg_(&pr_[tid]);
        // w_j = P(c, j) + conj(scale) u_j (j > c);  s_j = conj(P(c, j)) + scale t_j (j < c)
        wv[tid] = (tid > c) ? pc + conj_(scale) * sum : (tid < c ? conj_(pc) + scale * sum : zero_<T>());
      }
    }
    for (int r = r0 + tid; r < rows; r += NT) base[r + c * ld] = scale * base[r + c * ld];
    if (tid == 0 && lo <= c && c < hi) base[(c - lo) + c * ld] = sh_beta;
    __syncthreads();
    // ---- C: apply H^H to the remaining columns; column c of T (block 0)
    const T ctau = conj_(tau);
    if (grp < NG && jj > c) {
      const T wj = ctau * wv[jj];
      for (int r = max(0, c - lo) + grp; r < rows; r += NG) {
        const T vr = (lo + r == c) ? from_re<T>(1.0) : base[r + c * ld];
        base[r + jj * ld] -= vr * wj;
      }
    }
    if (blk == 0 && tid < b) {
      T val = zero_<T>();
      if (tid < c) {
        T acc = zero_<T>();
        for (int l = tid; l < c; ++l) acc += Tm[tid + l * b] * wv[l];
        val = -(tau * acc);
      } else if (tid == c) {
        val = tau;
      }
      Tm[tid + c * b] = val;
    }
    __syncthreads();
  }
  // ---- write back: R (upper part) into the panel with zeros below, Y explicitly
  for (int idx = tid; idx < rows * b; idx += NT) {
    const int r = idx % rows, j = idx / rows;
    const int pr = lo + r;
    const T val = base[r + j * ld];
    Y[pr + j * ldy] = (pr == j) ? from_re<T>(1.0) : (pr > j ? val : zero_<T>());
    P[pr + j * ldp] = (pr <= j) ? val : zero_<T>();
  }
}

// band[(i-j) + j*ldb] = A(i,j) for 0 <= i-j <= b, zero for b < i-j < ldb.
template <class T>
__global__ void k_extract_band(int n, int b, const T* A, long long lda, T* band, int ldb) {
  const long long total = (long long)n * ldb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int d = (int)(t % ldb), j = (int)(t / ldb);
    const int i = j + d;
    T v = zero_<T>();
    if (d <= b && i < n) v = A[i + j * lda];
    if (d == 0) v = from_re<T>(re_(v));
    band[t] = v;
  }
}

template <class T> size_t panel_smem(int R, int b, int use_smem) {
  size_t s = (size_t)(NT + b) * sizeof(T) + 32 * sizeof(double) + 64;
  if (use_smem) s += (size_t)(R | 1) * b * sizeof(T);
  return s;
}

}  // namespace

template <class T> int he2hb(Sys& s, T* A, int lda, int b) {
  const int n = s.n;
  GEV_TRY(allow_max_dyn_smem(k_panel_qr<T>));
  T* V1 = (T*)s.V1;
  // the panels' reflector columns are stored from their own first row on; the rows above are zero so
  // that consecutive panels form one wider compact-WY block in the back-transform
  GEV_CUDA_TRY(cudaMemsetAsync(V1, 0, sizeof(T) * (size_t)n * n, s.stream));
  T* T1 = (T*)s.T1;
  T* W0 = (T*)s.Pn;
  T* W1 = W0 + (size_t)n * 2 * s.b;
  T* sm0 = (T*)s.small;
  T* sm1 = sm0 + (size_t)s.b * s.b;
  double* nrm_part = (double*)s.panelws;     // 2 x 4096 (by column parity)
  T* prow = (T*)(nrm_part + 2 * 4096);        // 2 x b pivot rows
  T* w_part = prow + 2 * 128;                 // 2 x 4096 x b
  GridBar gb{(unsigned*)&s.status[ST_BARRIER_CNT], (unsigned*)&s.status[ST_BARRIER_GEN], s.status,
             &s.status[ST_ABORT]};
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zero = zero_<T>(), mhalf = from_re<T>(-0.5);
  int npanel = 0;
  for (int j0 = 0;; j0 += b) {
    const int r0 = j0 + b;
    const int m = n - r0;
    if (m < 2) break;
    ++npanel;
    T* Pp = A + r0 + (long long)j0 * lda;
    T* Yp = V1 + r0 + (long long)j0 * n;
    T* Tp = T1 + (long long)j0 * b;
    // ---- launch geometry: rows per block, shared-memory residency when it fits
    int per_sm = 1;
    int G = s.sms;
    int R = (m + G - 1) / G;
    if (R < 16) R = 16;
    G = (m + R - 1) / R;
    int use_smem = panel_smem<T>(R, b, 1) <= (size_t)200 * 1024 ? 1 : 0;
    size_t smem = panel_smem<T>(R, b, use_smem);
    GEV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_panel_qr<T>, NT, smem));
    if (per_sm < 1 || G > per_sm * s.sms) return GEV_ERR_UNSUPPORTED;
    if (G > 4096) return GEV_ERR_UNSUPPORTED;
    GEV_CUDA_TRY(cudaMemsetAsync(&s.status[ST_BARRIER_CNT], 0, 2 * sizeof(int), s.stream));
    int mm = m, bb = b;
    long long ldp = lda, ldy = n;
    void* args[] = {&mm, &bb, &Pp, &ldp, &Yp, &ldy, &Tp, &nrm_part, &w_part, &prow, &gb, &R, &use_smem};
    GEV_COUNT(s);
    GEV_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_panel_qr<T>, dim3(G), dim3(NT), args, smem, s.stream));
    // ---- two-sided update of the trailing block, the rank-2b update as ONE product:
    //      A22 -= Y V^H + V Y^H = [Y V] [V Y]^H  (K = 2b: the trailing block is read and written once)
    T* A22 = A + r0 + (long long)r0 * lda;
    T* YV = W1;                                // m x 2b: [Y | V]
    T* Wv = W1 + (size_t)n * b;                // its V half
    T* VY = W0 + (size_t)2 * n * 2 * s.b;      // m x 2b: [V | Y] (third panel buffer)
    gemm(s, gp<T>(m, b, m, 0, 0, one, A22, lda, Yp, n, zero, W0, n));  // W0 = A22 Y
    GemmP<T> g = gp<T>(m, b, b, 0, 0, one, W0, n, Tp, b, zero, Wv, n);   // W = W0 T
    g.tri_b = 2;
    gemm(s, g);
    gemm(s, gp<T>(b, b, m, 2, 0, one, Yp, n, Wv, n, zero, sm0, b));    // Z = Y^H W
    g = gp<T>(b, b, b, 2, 0, one, Tp, b, sm0, b, zero, sm1, b);         // U = T^H Z
    g.tri_a = 1;
    gemm(s, g);
    gemm(s, gp<T>(m, b, b, 0, 0, mhalf, Yp, n, sm1, b, one, Wv, n));   // V = W - Y U / 2
    GEV_TRY(copy2d<T>(s, m, b, Yp, n, YV, n));
    GEV_TRY(copy2d<T>(s, m, b, Wv, n, VY, n));
    GEV_TRY(copy2d<T>(s, m, b, Yp, n, VY + (size_t)n * b, n));
    g = gp<T>(m, m, 2 * b, 0, 2, mone, YV, n, VY, n, one, A22, lda);    // A22 -= [Y V] [V Y]^H
    g.c_lower = 1;
    gemm(s, g);
    GEV_TRY(mirror_lower<T>(s, m, A22, lda));
  }
  // ---- compact band for the bulge chasing
  const int ldb = 2 * b;
  if (ldb > s.ldband) return GEV_ERR_UNSUPPORTED;
  {
    long long total = (long long)n * ldb;
    unsigned blocks = cdiv(total, 256);
    if (blocks > 16u * s.sms) blocks = 16u * s.sms;
    GEV_COUNT(s);
    k_extract_band<T><<<blocks, 256, 0, s.stream>>>(n, b, A, lda, (T*)s.band, ldb);
    GEV_TRY(last_error());
  }
  s.band_b_used = b;
  s.have_band = true;
  s.have_tridiag_refl = false;
  s.nsbr_panels = npanel;
  s.q1_pw = b;
  s.q1_off = b;
  s.q1_nrefl = npanel * b;
  s.one_stage_used = false;
  return 0;
}

// Y <- Q1 Y (n x k), Q1 = Q_0 Q_1 ... Q_last: the panels' compact-WY blocks, applied G panels at a
// time.  Panel p holds reflectors p*pw .. p*pw + w_p - 1 (w_p = pw but for a narrower last panel of
// the one-stage reduction), stored in those columns of V1 from row p*pw + off on (off = b for the
// full -> band panels, 1 for the one-stage ones), each zero above its own first row (V1 is cleared
// before the reduction), with its w_p x w_p factor T_p at T1 + p pw^2 (ld pw).  Consecutive panels
// p .. p+G-1 merge into one block  Q_p ... Q_{p+G-1} = I - Yg Tg Yg^H,  Yg = [Y_p ... Y_{p+G-1}],
// Tg upper triangular, built block column by block column from the T_j and the Gram blocks Yg^H Yg:
//     Tg(0:o_j, o_j:o_j+w_j) = -Tg(0:o_j, 0:o_j) (Yg(:, 0:o_j)^H Y_j) T_j,   Tg(o_j.., o_j..) = T_j.
// Each group then costs three products with inner dimension sum w_j (or m), last group first.
template <class T> int bt_he2hb(Sys& s, T* Yb, int ldy, int k) {
  const int n = s.n, pw = s.q1_pw, off = s.q1_off, nrefl = s.q1_nrefl;
  T* V1 = (T*)s.V1;
  T* T1 = (T*)s.T1;
  const int np = s.nsbr_panels;
  if (np <= 0) return 0;
  const int G = std::min(4, np);
  const int gb = G * pw;                  // <= 4 b
  T* Wk = (T*)s.Pn;                       // gb x k  (the panel buffers: 8 b n elements)
  T* Wk2 = Wk + (size_t)gb * k;           // gb x k
  T* Tg = (T*)s.btg;                      // gb x gb
  T* Gg = Tg + (size_t)gb * gb;           // gb x gb Gram blocks
  T* Xg = Gg + (size_t)gb * gb;           // gb x pw
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zero = zero_<T>();
  auto width = [&](int p) { return std::min(pw, nrefl - p * pw); };
  const int ngroups = (np + G - 1) / G;
  for (int q = ngroups - 1; q >= 0; --q) {
    const int p0 = q * G, pc = std::min(G, np - p0);
    int w = 0;
    for (int j = 0; j < pc; ++j) w += width(p0 + j);
    const int j0 = p0 * pw, r0 = j0 + off, m = n - r0;
    if (m <= 0 || w <= 0) continue;
    const T* Yg = V1 + r0 + (long long)j0 * n;  // m x w
    // Tg: block column 0 = T_p0; block column j from the Gram blocks
    GEV_CUDA_TRY(cudaMemset2DAsync(Tg, sizeof(T) * gb, 0, sizeof(T) * w, w, s.stream));
    GEV_TRY(copy2d<T>(s, width(p0), width(p0), T1 + (size_t)p0 * pw * pw, pw, Tg, gb));
    if (pc > 1) {
      GemmP<T> g = gp<T>(w, w, m, 2, 0, one, Yg, n, Yg, n, zero, Gg, gb);  // Gram Yg^H Yg
      gemm(s, g);
      for (int j = 1; j < pc; ++j) {
        const int oj = j * pw, wj = width(p0 + j);
        const T* Tj = T1 + (size_t)(p0 + j) * pw * pw;
        g = gp<T>(oj, wj, wj, 0, 0, one, Gg + (size_t)oj * gb, gb, Tj, pw, zero, Xg, gb);  // X = G(0:oj, j) T_j
        g.tri_b = 2;
        gemm(s, g);
        g = gp<T>(oj, wj, oj, 0, 0, mone, Tg, gb, Xg, gb, zero, Tg + (size_t)oj * gb, gb);
        g.tri_a = 2;                                                   // Tg(0:oj, j) = -Tg(0:oj, 0:oj) X
        gemm(s, g);
        GEV_TRY(copy2d<T>(s, wj, wj, Tj, pw, Tg + oj + (size_t)oj * gb, gb));
      }
    }
    T* Ysub = Yb + r0;
    gemm(s, gp<T>(w, k, m, 2, 0, one, Yg, n, Ysub, ldy, zero, Wk, gb));  // Wk = Yg^H Y
    GemmP<T> g = gp<T>(w, k, w, 0, 0, one, Tg, gb, Wk, gb, zero, Wk2, gb);  // Wk2 = Tg Wk
    g.tri_a = 2;
    gemm(s, g);
    gemm(s, gp<T>(m, k, w, 0, 0, mone, Yg, n, Wk2, gb, one, Ysub, ldy));  // Y -= Yg Wk2
  }
  return last_error();
}

// Step 6 ("Back"): Y = Q1 Q2 D Z.
template <class T> int back(Sys& s, const double* Z, int ldz, int k, T* Y, int ldy) {
  if (s.one_stage_used) return back_td<T>(s, Z, ldz, k, Y, ldy);
  GEV_TRY(bt_hb2st<T>(s, Z, ldz, k, Y, ldy));
  GEV_TRY(bt_he2hb<T>(s, Y, ldy, k));
  return 0;
}

template int back<double>(Sys&, const double*, int, int, double*, int);
template int back<zd>(Sys&, const double*, int, int, zd*, int);
template int he2hb<double>(Sys&, double*, int, int);
template int he2hb<zd>(Sys&, zd*, int, int);
template int bt_he2hb<double>(Sys&, double*, int, int);
template int he2hb<float>(Sys&, float*, int, int);
template int bt_he2hb<float>(Sys&, float*, int, int);
template int bt_he2hb<zd>(Sys&, zd*, int, int);

}  // namespace gev
