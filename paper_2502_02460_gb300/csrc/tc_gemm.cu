// FP32 matrix products from BF16 split products on the 5th-generation tensor cores (tcgen05,
// kind::f16, FP32 accumulation in tensor memory), for the FP32 stages of the mixed form.
//
//   x = x1 + x2 + x3 with x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2)  (each step exact
//   in FP32, so x1 + x2 + x3 carries 24 significant bits: the FP32 value itself)
//   a b ~ sum over the pairs (p, q) with p + q <= 4 of a_p b_q:
//     BF16x6: a1b1 + a1b2 + a2b1 + a1b3 + a2b2 + a3b1  (dropped terms at most 2^-23 |a b|: FP32 level)
//     BF16x3: a1b1 + a1b2 + a2b1                        (about 16 significant bits)
//   all products of one output accumulate in one FP32 tensor-memory accumulator.
//
// Data flow as in the emulated FP64 product (ozaki.cu): a split pass writes the three BF16 planes of
// op(A) and op(B) to global memory in the order the MMAs consume them (one 16-deep k-slice of a
// 128-row A tile = 3 planes x 4 KB; of a 256-column B tile = 3 x 8 KB), the GEMM kernel moves them
// with bulk asynchronous copies into a 6-stage shared-memory ring, warp 9 issues the 128 x 256 x 16
// MMAs, warps 0-7 read the accumulator (one TMEM lane per output row, half of the 256 columns each)
// and write C.  Every mbarrier wait is bounded; on expiry the kernel records ST_TIMEOUT, waits
// (bounded) for its copies and MMAs in flight, frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "tcgen05.cuh"

namespace gev {

namespace {

using namespace tc;

constexpr int TM = 128, TN = 256, KS = 16, NSTAGE = 6, NPL = 3;
constexpr int A_PL = TM * KS * 2;          // one plane of a 128 x 16 slice: 4 KB
constexpr int B_PL = TN * KS * 2;          // one plane of a 256 x 16 slice: 8 KB
constexpr int A_ST = NPL * A_PL;           // 12 KB
constexpr int B_ST = NPL * B_PL;           // 24 KB
constexpr int STAGE = A_ST + B_ST;         // 36 KB
constexpr int SMEM_TC = NSTAGE * STAGE + 1024;
constexpr int NEPI_W = 8;                  // epilogue warps: TMEM lanes 32 (w % 4), columns 128 (w / 4)
constexpr int HC = TN / 2;
constexpr int NTH = 32 * (NEPI_W + 2);     // + copy warp 8 + MMA warp 9
constexpr int TMEM_COLS = 256;
constexpr int GROUP_M = 8;

// three BF16 planes of one operand (vector r, element k; rows padded to RT tiles of TR, k to KT
// slices of 16).  One thread per (r, 8 consecutive k): 16 bytes to each plane.
template <class TI>
__global__ void k_split3(int R, int K, const TI* X, long long sr, long long sk, int keep, int TR, int RT, int KT,
                         unsigned char* out) {
  const long long Rp = (long long)RT * TR, G = 2LL * KT;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= Rp * G) return;
  long long r, g;
  if (sr == 1) { r = t % Rp; g = t / Rp; } else { g = t % G; r = t / G; }
  uint32_t pk[NPL][4];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    uint16_t h[2][NPL];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const long long k = g * 8 + q + u;
      float x = 0.f;
      if (r < R && k < K && kept(keep, r, k)) x = (float)X[r * sr + k * sk];
      const __nv_bfloat16 x1 = __float2bfloat16_rn(x);
      const float r1 = x - __bfloat162float(x1);  // exact
      const __nv_bfloat16 x2 = __float2bfloat16_rn(r1);
      const float r2 = r1 - __bfloat162float(x2);  // exact
      const __nv_bfloat16 x3 = __float2bfloat16_rn(r2);
      h[u][0] = __bfloat16_as_ushort(x1);
      h[u][1] = __bfloat16_as_ushort(x2);
      h[u][2] = __bfloat16_as_ushort(x3);
    }
#pragma unroll
    for (int p = 0; p < NPL; ++p) pk[p][q / 2] = (uint32_t)h[0][p] | ((uint32_t)h[1][p] << 16);
  }
  const long long rt = r / TR, kt = g >> 1;
  const int plane_bytes = TR * KS * 2;
  unsigned char* base =
      out + ((rt * KT + kt) * NPL) * (long long)plane_bytes + toff16((int)(r % TR), (int)(g & 1) * 8);
#pragma unroll
  for (int p = 0; p < NPL; ++p)
    *reinterpret_cast<uint4*>(base + (long long)p * plane_bytes) = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
}

struct TcP {
  int M, N, K, c_lower, tri_a, tri_b;
  int MT, NT, KT, ksplit, nprod, c_f64;
  float alpha, beta;
  void* C;
  long long ldc;
  float* ws;  // split-K partials: ws[z M N + i + j M]
  const unsigned char* Ap;
  const unsigned char* Bp;
  int* status;
  int nstage;  // stages of the shared-memory ring (<= NSTAGE; the launch's dynamic shared memory)
  // block-diagonal op(A) (0: off): block j has rows [j bd_bm, (j+1) bd_bm) and its non-zero columns
  // [j bd_bk, (j+1) bd_bk); the A planes then hold, per row tile, only that tile's K range (compact)
  int bd_bm, bd_bk;
};

// K slices of a row tile of a block-diagonal op(A): the first slice of the tile's K range and the
// count (bm, bk multiples of 16 that divide / are multiples of the 128-row tile)
__host__ __device__ __forceinline__ void bd_range32(int bm, int bk, int mt, int* first, int* count) {
  if (bm <= TM) {
    const int per = TM / bm;
    *first = mt * per * bk / KS;
    *count = per * bk / KS;
  } else {
    *first = (mt / (bm / TM)) * bk / KS;
    *count = bk / KS;
  }
}

// Entry (i, kk) of a real block-diagonal back-transform-2 operand in FP32 (BdOp, common.cuh).
__device__ __forceinline__ float bd_at32(const BdOp& o, long long i, long long kk) {
  const int b = o.b;
  if (o.kind == 1) {  // V_j^H: row q of block j, column r of the block's window
    const long long j = i / b, q = i % b, r = kk - 2LL * b * j;
    if (r < 0 || r >= 2 * b || j >= o.nblk) return 0.f;
    const long long g = o.g_lo + j, t = o.L - (o.ngroups - 1 - g), sw = g * b + q, rel = r - q;
    if (sw > o.n - 3 || rel < 0 || rel >= b || o.w00 + 2LL * b * j + r >= o.n) return 0.f;
    const long long rid = sw * o.ntask + t;
    if (static_cast<const float*>(o.tau2)[rid] == 0.f) return 0.f;
    return static_cast<const float*>(o.V2)[rid * b + rel];
  }
  const long long j = i / (2 * b), r = i % (2 * b), q = kk - (long long)b * j;  // W_j: row r, column q
  if (q < 0 || q >= b || j >= o.nblk) return 0.f;
  return static_cast<const float*>(o.W)[j * 2LL * b * b + r + q * 2LL * b];
}

// The three BF16 planes of a block-diagonal op(A) in the compact layout (row tile mt holds only the
// slices of its K range).  One warp per row of the padded MT x 128 rows; lane l takes 8 consecutive
// columns of the range and writes 16 bytes to each plane.
__global__ void k_split3_bd(int M, BdOp o, int bm, int bk, int MT, unsigned char* out) {
  const long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= (long long)MT * TM) return;
  const int mt = (int)(i / TM);
  int f = 0, c = 0;
  bd_range32(bm, bk, mt, &f, &c);
  if (lane * 8 >= c * KS) return;
  uint32_t pk[NPL][4];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    uint16_t h[2][NPL];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const long long kk = (long long)f * KS + lane * 8 + q + u;
      const float x = (i < M) ? bd_at32(o, i, kk) : 0.f;
      const __nv_bfloat16 x1 = __float2bfloat16_rn(x);
      const float r1 = x - __bfloat162float(x1);  // exact
      const __nv_bfloat16 x2 = __float2bfloat16_rn(r1);
      const float r2 = r1 - __bfloat162float(x2);  // exact
      const __nv_bfloat16 x3 = __float2bfloat16_rn(r2);
      h[u][0] = __bfloat16_as_ushort(x1);
      h[u][1] = __bfloat16_as_ushort(x2);
      h[u][2] = __bfloat16_as_ushort(x3);
    }
#pragma unroll
    for (int p = 0; p < NPL; ++p) pk[p][q / 2] = (uint32_t)h[0][p] | ((uint32_t)h[1][p] << 16);
  }
  const int plane_bytes = TM * KS * 2;
  unsigned char* base = out + (((long long)mt * c + (lane >> 1)) * NPL) * plane_bytes + toff16((int)(i % TM), (lane & 1) * 8);
#pragma unroll
  for (int p = 0; p < NPL; ++p)
    *reinterpret_cast<uint4*>(base + (long long)p * plane_bytes) = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
}

__global__ void __launch_bounds__(NTH, 1) tc32_kernel(TcP p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int per_group = GROUP_M * p.NT;
  const int first = (blockIdx.x / per_group) * GROUP_M;
  const int gm = min(p.MT - first, GROUP_M);
  const int within = blockIdx.x % per_group;
  const int mt = first + within % gm, nt = within / gm;
  const int m0 = mt * TM, n0 = nt * TN;
  if (p.c_lower && n0 > m0 + TM - 1) return;
  long long kb, ke;
  tile_k_range(p.tri_a, p.tri_b, m0, TM, n0, TN, p.K, 0, kb, ke);
  int s_lo = (int)(kb > 0 ? kb / KS : 0), s_hi = (int)(ke > 0 ? (ke + KS - 1) / KS : 0);
  if (s_hi < s_lo) s_hi = s_lo;
  // A-plane slices: a_kt per row tile, slice kt read at kt - a_off
  int a_kt = p.KT, a_off = 0;
  if (p.bd_bm) {
    int f = 0, c = 0;
    bd_range32(p.bd_bm, p.bd_bk, mt, &f, &c);
    s_lo = min(f, p.KT);
    s_hi = min(f + c, p.KT);
    a_kt = c;
    a_off = f;
  }
  const int nstage = p.nstage;
  if (p.ksplit > 1) {
    const int tot = s_hi - s_lo, z = blockIdx.y;
    const int a = s_lo + (int)((long long)tot * z / p.ksplit);
    const int b = s_lo + (int)((long long)tot * (z + 1) / p.ksplit);
    s_lo = a;
    s_hi = b;
  }
  const int nst = s_hi - s_lo;

  unsigned char* ctrl = smem + nstage * STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(ctrl);
  uint64_t* empty = full + NSTAGE;
  uint64_t* accd = empty + NSTAGE;  // accumulator complete
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ctrl + 256);
  volatile int* err = reinterpret_cast<volatile int*>(ctrl + 320);
  int* issued = reinterpret_cast<int*>(ctrl + 384);
  int* consumed = reinterpret_cast<int*>(ctrl + 448);
  if (tid == 0) {
    for (int s = 0; s < nstage; ++s) {
      mbar_init(su32(&full[s]), 1);
      mbar_init(su32(&empty[s]), 1);
    }
    mbar_init(su32(accd), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *err = 0;
    *issued = 0;
    *consumed = 0;
  }
  if (warp == 0) tmem_alloc(su32(tslot), TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (warp == NEPI_W) {
    // ---- copy warp
    if (lane == 0) {
      const unsigned char* a_src = p.Ap + ((long long)mt * a_kt - a_off) * A_ST;
      const unsigned char* b_src = p.Bp + (long long)nt * p.KT * B_ST;
      for (int s = 0; s < nst; ++s) {
        const int slot = s % nstage;
        if (s >= nstage && !bar_wait(su32(&empty[slot]), ((s / nstage) - 1) & 1, err)) {
          if (!*err) *err = 421;
          break;
        }
        const uint32_t fb = su32(&full[slot]);
        mbar_expect_tx(fb, STAGE);
        const uint32_t dst = su32(smem + slot * STAGE);
        const long long kt = s_lo + s;
        bulk_g2s(dst, a_src + kt * A_ST, A_ST, fb);
        bulk_g2s(dst + A_ST, b_src + kt * B_ST, B_ST, fb);
        *issued = s + 1;
      }
    }
  } else if (warp == NEPI_W + 1) {
    // ---- MMA warp: 6 (or 3) split products per 16-deep slice into one accumulator
    if (lane == 0) {
      const uint32_t id = idesc_bf16(TM, TN);
      for (int s = 0; s < nst; ++s) {
        const int slot = s % nstage;
        if (!bar_wait(su32(&full[slot]), (s / nstage) & 1, err)) {
          if (!*err) *err = 422;
          break;
        }
        *consumed = s + 1;
        fence_after();
        const uint32_t a0 = su32(smem + slot * STAGE), b0 = a0 + A_ST;
        // pairs in order of decreasing magnitude: (1,1) (1,2) (2,1) [(1,3) (2,2) (3,1)]
        mma_bf16(tmem, sdesc16(a0), sdesc16(b0), id, s > 0 ? 1 : 0);
        mma_bf16(tmem, sdesc16(a0), sdesc16(b0 + B_PL), id, 1);
        mma_bf16(tmem, sdesc16(a0 + A_PL), sdesc16(b0), id, 1);
        if (p.nprod == 6) {
          mma_bf16(tmem, sdesc16(a0), sdesc16(b0 + 2 * B_PL), id, 1);
          mma_bf16(tmem, sdesc16(a0 + A_PL), sdesc16(b0 + B_PL), id, 1);
          mma_bf16(tmem, sdesc16(a0 + 2 * A_PL), sdesc16(b0), id, 1);
        }
        commit(su32(&empty[slot]));
      }
      commit(su32(accd));
    }
  } else {
    // ---- epilogue warps
    bool good = true;
    if (nst > 0 && !bar_wait(su32(accd), 0, err)) {
      good = false;
      if (!*err) *err = 423;
    }
    const bool any = good && nst > 0;
    fence_after();
    const int quarter = warp & 3, col0 = (warp >> 2) * HC;
    const int gi = m0 + quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
    for (int cb = 0; cb < HC; cb += 16) {
      uint32_t r[16];
      if (any) {
        tmem_ld16(lane_base + (uint32_t)cb, r);
        tmem_wait_ld();
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = 0u;
      }
      if (gi < p.M) {
        const bool read_c = p.ksplit == 1 && p.beta != 0.f;
#pragma unroll
        for (int h = 0; h < 16; h += 8) {
          // the loads of 8 outputs first, so that they overlap
          double cin[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int gj = n0 + col0 + cb + h + u;
            const bool ok = gj < p.N && !(p.c_lower && gi < gj);
            cin[u] = 0.0;
            if (ok && read_c)
              cin[u] = p.c_f64 ? static_cast<const double*>(p.C)[gi + gj * p.ldc]
                               : (double)static_cast<const float*>(p.C)[gi + gj * p.ldc];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int gj = n0 + col0 + cb + h + u;
            if (gj >= p.N || (p.c_lower && gi < gj)) continue;
            const float v = __uint_as_float(r[h + u]);
            if (p.ksplit > 1) {
              p.ws[(long long)blockIdx.y * p.M * p.N + gi + (long long)gj * p.M] = v;
            } else if (p.c_f64) {
              const double o = (double)p.alpha * (double)v;
              static_cast<double*>(p.C)[gi + gj * p.ldc] = read_c ? o + (double)p.beta * cin[u] : o;
            } else {
              const float o = p.alpha * v;
              static_cast<float*>(p.C)[gi + gj * p.ldc] = read_c ? o + p.beta * (float)cin[u] : o;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0 && *err) {
    // a wait gave up: let the copies already issued land before the shared memory is released
    for (int s = *consumed; s < *issued; ++s) bar_wait_plain(su32(&full[s % nstage]), (s / nstage) & 1);
    atomicCAS(&p.status[ST_TIMEOUT], 0, *err);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// C = alpha sum_z ws[z] + beta C in a fixed order (deterministic)
template <class TO>
__global__ void k_tc_reduce(int M, int N, int ks, int c_lower, float alpha, const float* ws, float beta, TO* C,
                            long long ldc) {
  const long long total = (long long)M * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % M), j = (int)(t / M);
    if (c_lower && i < j) continue;
    float s = 0.f;
    for (int z = 0; z < ks; ++z) s += ws[(long long)z * total + t];
    TO* c = &C[i + (long long)j * ldc];
    const TO o = (TO)alpha * (TO)s;
    *c = (beta != 0.f) ? o + (TO)beta * (*c) : o;
  }
}

size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

size_t gemm_tc32_scratch(int M, int N, int K) {
  const size_t Mp = rup(std::max(M, 1), TM), Np = rup(std::max(N, 1), TN), Kp = rup(std::max(K, 1), KS);
  return rup(Mp * Kp * 2 * NPL, 256) + Np * Kp * 2 * NPL;
}

// C = alpha op(A) op(B) + beta C with FP32 products formed from BF16 splits (nprod 6 or 3); the
// split planes live in s.ozws (s.ozws_bytes >= gemm_tc32_scratch).  Returns false (nothing
// launched) when the scratch is too small.
template <class TI, class TO>
bool gemm_tc32(Sys& s, const GemmP<TI>& q, TO* C, float alpha, float beta, int nprod) {
  if (q.M <= 0 || q.N <= 0) return true;
  if (!s.ozws || gemm_tc32_scratch(q.M, q.N, q.K) > s.ozws_bytes) return false;
  if (allow_dyn_smem(tc32_kernel, SMEM_TC) != 0) return false;  // the caller takes the CUDA-core product
  const size_t Mp = rup(q.M, TM), Kp = rup(std::max(q.K, 1), KS);
  unsigned char* Ap = static_cast<unsigned char*>(s.ozws);
  unsigned char* Bp = Ap + rup(Mp * Kp * 2 * NPL, 256);
  const int MT = (int)(Mp / TM), NT = (int)(rup(q.N, TN) / TN), KT = (std::max(q.K, 0) + KS - 1) / KS;
  // op(A) row i, element k: A[i + k lda] (ta 0) or A[k + i lda]; op(B) column j, element k:
  // B[k + j ldb] (tb 0) or B[j + k ldb]
  const long long a_sr = q.ta ? q.lda : 1, a_sk = q.ta ? 1 : q.lda;
  const long long b_sr = q.tb ? 1 : q.ldb, b_sk = q.tb ? q.ldb : 1;
  const int keep_a = q.tri_a == 1 ? 1 : (q.tri_a == 2 ? 2 : 0);
  const int keep_b = q.tri_b == 1 ? 2 : (q.tri_b == 2 ? 1 : 0);
  if (KT > 0) {
    GEV_COUNT(s);
    k_split3<TI><<<cdiv((long long)MT * TM * 2 * KT, 256), 256, 0, s.stream>>>(q.M, q.K, q.A, a_sr, a_sk, keep_a,
                                                                              TM, MT, KT, Ap);
    GEV_COUNT(s);
    k_split3<TI><<<cdiv((long long)NT * TN * 2 * KT, 256), 256, 0, s.stream>>>(q.N, q.K, q.B, b_sr, b_sk, keep_b,
                                                                              TN, NT, KT, Bp);
  }
  TcP p{};
  p.M = q.M; p.N = q.N; p.K = std::max(q.K, 0); p.c_lower = q.c_lower; p.tri_a = q.tri_a; p.tri_b = q.tri_b;
  p.MT = MT; p.NT = NT; p.KT = KT; p.nprod = nprod; p.c_f64 = std::is_same<TO, double>::value ? 1 : 0;
  p.alpha = alpha; p.beta = beta; p.C = C; p.ldc = q.ldc; p.Ap = Ap; p.Bp = Bp; p.status = s.status;
  p.nstage = NSTAGE;
  long long tiles = (long long)MT * NT;
  if (q.c_lower) tiles = (tiles + MT) / 2;
  int ks = 1;
  if (tiles < s.sms && KT >= 64) {
    ks = (int)std::min<long long>((2LL * s.sms + tiles - 1) / tiles, KT / 32);
    ks = std::min(ks, 16);
    while (ks > 1 && (size_t)ks * q.M * q.N * sizeof(float) > s.splitws_bytes) --ks;
  }
  p.ksplit = ks;
  p.ws = ks > 1 ? static_cast<float*>(s.splitws) : nullptr;
  GEV_COUNT(s);
  tc32_kernel<<<dim3(MT * NT, ks), NTH, SMEM_TC, s.stream>>>(p);
  if (ks > 1) {
    unsigned blocks = cdiv((long long)q.M * q.N, 256);
    if (blocks > 8u * s.sms) blocks = 8u * s.sms;
    GEV_COUNT(s);
    k_tc_reduce<TO><<<blocks, 256, 0, s.stream>>>(q.M, q.N, ks, q.c_lower, alpha, p.ws, beta, C, q.ldc);
  }
  return true;
}

namespace {

struct BdLayout32 {
  size_t a_off, b_off, total;
  int MT, NT, KT, acount;
};

BdLayout32 bd_layout32(int M, int N, int K, int bm, int bk) {
  BdLayout32 L;
  L.MT = (int)(rup(std::max(M, 1), TM) / TM);
  L.NT = (int)(rup(std::max(N, 1), TN) / TN);
  L.KT = (std::max(K, 1) + KS - 1) / KS;
  int f = 0;
  bd_range32(bm, bk, 0, &f, &L.acount);
  L.a_off = 0;
  L.b_off = rup((size_t)L.MT * L.acount * A_ST, 256);
  L.total = L.b_off + (size_t)L.NT * L.KT * B_ST;
  return L;
}

}  // namespace

size_t gemm_f32_bdiag_scratch(int M, int N, int K, int bm, int bk) { return bd_layout32(M, N, K, bm, bk).total; }

// C (M x N) = alpha op(A) B + beta C in FP32, op(A) a real block-diagonal operand (BdOp with FP32
// data, blocks bm x bk), from BF16x6 split products; each output tile reads only its K range (4 or
// 16 slices).  A three-stage ring keeps two CTAs on an SM (shared memory 109 KB, tensor memory 256
// columns each), so one CTA's epilogue overlaps the other's products.
bool gemm_f32_bdiag(Sys& s, int M, int N, int K, const BdOp& a, int bm, int bk, const float* B, long long ldb,
                    float alpha, float beta, float* C, long long ldc) {
  if (M <= 0 || N <= 0) return true;
  const BdLayout32 L = bd_layout32(M, N, K, bm, bk);
  if (!s.ozws || L.total > s.ozws_bytes) return false;
  if (allow_dyn_smem(tc32_kernel, SMEM_TC) != 0) return false;
  unsigned char* Ap = static_cast<unsigned char*>(s.ozws) + L.a_off;
  unsigned char* Bp = static_cast<unsigned char*>(s.ozws) + L.b_off;
  GEV_COUNT(s);
  k_split3_bd<<<cdiv((long long)L.MT * TM * 32, 256), 256, 0, s.stream>>>(M, a, bm, bk, L.MT, Ap);
  if (K > 0) {
    GEV_COUNT(s);
    k_split3<float><<<cdiv((long long)L.NT * TN * 2 * L.KT, 256), 256, 0, s.stream>>>(N, K, B, ldb, 1, 0, TN, L.NT,
                                                                                   L.KT, Bp);
  }
  TcP p{};
  p.M = M; p.N = N; p.K = std::max(K, 0); p.c_lower = 0; p.tri_a = 0; p.tri_b = 0;
  p.MT = L.MT; p.NT = L.NT; p.KT = L.KT; p.nprod = s.fp32_tc == 3 ? 3 : 6; p.c_f64 = 0;
  p.alpha = alpha; p.beta = beta; p.C = C; p.ldc = ldc; p.Ap = Ap; p.Bp = Bp; p.status = s.status;
  p.ksplit = 1;
  p.ws = nullptr;
  p.bd_bm = bm;
  p.bd_bk = bk;
  p.nstage = std::min(3, L.acount);  // 109 KB of shared memory: two CTAs per SM
  GEV_COUNT(s);
  tc32_kernel<<<dim3(L.MT * L.NT, 1), NTH, (size_t)p.nstage * STAGE + 1024, s.stream>>>(p);
  return true;
}

template bool gemm_tc32<float, float>(Sys&, const GemmP<float>&, float*, float, float, int);
template bool gemm_tc32<float, double>(Sys&, const GemmP<float>&, double*, float, float, int);
template bool gemm_tc32<double, double>(Sys&, const GemmP<double>&, double*, float, float, int);
template bool gemm_tc32<double, float>(Sys&, const GemmP<double>&, float*, float, float, int);

}  // namespace gev

extern "C" size_t gev_gemm_f32_scratch_bytes(int M, int N, int K) {
  if (M < 0 || N < 0 || K < 0) return 0;
  return ((gev::gemm_tc32_scratch(M, N, K) + 255) & ~(size_t)255) + ((size_t)16 << 20);
}

extern "C" int gev_gemm_f32(int M, int N, int K, int ta, int tb, float alpha, const float* A, int lda,
                            const float* B, int ldb, float beta, float* C, int ldc, int engine, void* stream,
                            int* status_dev, void* scratch_dev, size_t scratch_bytes) {
  using namespace gev;
  if (M < 0) return -1;
  if (N < 0) return -2;
  if (K < 0) return -3;
  if (ta < 0 || ta > 1) return -4;
  if (tb < 0 || tb > 1) return -5;
  if (!A && M > 0 && K > 0) return -7;
  if (lda < std::max(1, ta ? K : M)) return -8;
  if (!B && K > 0 && N > 0) return -9;
  if (ldb < std::max(1, tb ? N : K)) return -10;
  if (!C && M > 0 && N > 0) return -12;
  if (ldc < std::max(1, M)) return -13;
  if (engine < 0 || engine > 2) return -14;
  if (!status_dev) return -16;
  if (engine > 0 && (!scratch_dev || scratch_bytes < gev_gemm_f32_scratch_bytes(M, N, K))) return -17;
  Sys s;
  s.stream = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  GEV_CUDA_TRY(cudaGetDevice(&dev));
  GEV_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  s.sms = sms > 0 ? sms : 152;
  s.status = status_dev;
  GemmP<float> g = gp<float>(M, N, K, ta, tb, alpha, A, lda, B, ldb, beta, C, ldc);
  if (engine == 0) {
    s.splitws = nullptr;
    s.splitws_bytes = 0;
    gemm32<float, float>(s, g, C, alpha, beta);
  } else {
    const size_t planes = (gemm_tc32_scratch(M, N, K) + 255) & ~(size_t)255;
    s.ozws = scratch_dev;
    s.ozws_bytes = planes;
    s.splitws = static_cast<unsigned char*>(scratch_dev) + planes;
    s.splitws_bytes = scratch_bytes - planes;
    s.fp32_tc = 0;  // gemm_tc32 directly, no size policy
    if (!gemm_tc32<float, float>(s, g, C, alpha, beta, engine == 1 ? 6 : 3)) return GEV_ERR_CUDA;
  }
  GEV_TRY(last_error());
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  return 0;
}
