// FP64 GEMM emulated on the BF16 tensor cores (tcgen05), for the FP64 matrix products.
//
// GB300 executes FP64 at ~1 TFLOP/s (DMMA and DFMA alike) but BF16 at ~1.9 PFLOP/s, so an FP64
// product is formed from exact BF16 pieces (an error-free splitting in the manner of Ozaki, Ogita,
// Oishi and Rump):
//
//   row i of op(A) is scaled by 2^-(E_i+1), column j of op(B) by 2^-(F_j+1) (E, F: the smallest
//   exponents with |x| < 2^E over the row / column), so every scaled entry lies in (-1/2, 1/2);
//   X = x 2^(55-E) truncated to an integer (|X| < 2^55) is written in balanced radix 2^7,
//   X = sum_{p=1..8} a_p 2^(56-7p) with integer digits |a_p| <= 64 (integer arithmetic only), and
//   a_p 2^-7p is stored as BF16, exactly.
//
//   A B = 2^(E_i+F_j+2) sum_{p,q} (a_p 2^-7p)(b_q 2^-7q); pairs with p + q >= 10 (each below 2^-58
//   of the scale) are dropped.  For d = p + q <= 7 the products of diagonal d are integers times
//   2^-7d of magnitude <= 2^12; summed over a K chunk of 512 with at most 6 pairs they stay below
//   2^24, so the FP32 tensor-memory accumulator holds them exactly.  After each chunk the six exact
//   sums are added, as integers in units of 2^-49, to one 64-bit integer accumulator per output
//   (exact; integer operations are cheap on GB300 while FP64 additions are not).  The diagonals
//   d = 8, 9 share one FP32 accumulator over all of K; its roundings stay near 2^-51 of the scale.
//
// Data flow: a split pass writes the 8 digit planes of op(A) and op(B) to global memory in the
// order the MMAs consume them (one 16-deep k-slice of a 128-row A tile = 8 planes x 4 KB,
// contiguous; of a 64-column B tile = 8 x 2 KB), so the GEMM kernel moves them with plain bulk
// asynchronous copies into a 4-stage shared-memory ring.  Warp roles: warp 8 issues the copies,
// warp 9 issues the 36 MMAs per slice (tcgen05, accumulators in TMEM: 6 exact diagonals + 1
// shared, 64 columns each), warps 0-7 (one TMEM lane per output row, half of its 64 columns
// each) drain the exact accumulators at every chunk end and write C.  Every mbarrier wait is bounded; on expiry the kernel records
// ST_TIMEOUT, waits (bounded) for its copies and MMAs in flight, frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "tcgen05.cuh"

namespace gev {

namespace {

using namespace tc;

constexpr int OM = 128, ON = 64, KS = 16, NSTAGE = 4, NSLICE = 8, DMAX = 9, DEXACT = 7;
constexpr int CHUNK = 32;                  // k-slices per exact chunk (512 of K)
constexpr int KMAX = 32768;                // K per launch: the int64 sums stay below 2^63
constexpr int A_TILE = OM * KS * 2;        // one plane of a 128 x 16 slice: 4 KB
constexpr int B_TILE = ON * KS * 2;        // one plane of a 64 x 16 slice: 2 KB
constexpr int A_STAGE = NSLICE * A_TILE;   // 32 KB
constexpr int B_STAGE = NSLICE * B_TILE;   // 16 KB
constexpr int STAGE = A_STAGE + B_STAGE;   // 48 KB
constexpr int SMEM_OZ = NSTAGE * STAGE + 1024;
constexpr int NEPI_W = 8;                  // epilogue warps: TMEM lanes 32 (w % 4), columns 32 (w / 4)
constexpr int HC = ON / 2;                  // output columns per epilogue thread
constexpr int NTH = 32 * (NEPI_W + 2);      // + copy warp 8 + MMA warp 9
constexpr int TMEM_COLS_OZ = 512;
constexpr int SHARED_SLOT = DEXACT - 1;    // TMEM slot of d = 8, 9; exact d at slot d - 2
constexpr int GROUP_M = 16;                // raster: 16 row tiles share their B slices in L2
constexpr int EXP_BAD = 1 << 20;           // exponent marking a non-finite entry
constexpr int EXP_ZERO = -4000;            // exponent of an all-zero vector

// exponent e with |x| < 2^e for a finite x != 0; EXP_ZERO for 0, EXP_BAD for Inf / NaN
__device__ __forceinline__ int exp_above(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7FF);
  if (be == 0x7FF) return EXP_BAD;
  if (be == 0) return (b << 1) ? -1022 : EXP_ZERO;
  return be - 1022;
}


// One operand of a product as the exponent and split passes see it: vectors r (rows of op(A) or
// columns of op(B)) of elements k.  Real data: element (r, k) at X[r sr + k sk].  Complex data
// (double2 elements, strides in elements) enters through the real embedding of C = op(A) op(B):
//   cx 1 (A side): vector r = 2i + a, element k = 2l + b of the 2 x 2 block [[x, -y], [y, x]] of
//                  op(A)_il = x + iy;
//   cx 2 (B side): vector j, element k = 2l + c: x (c = 0) or y (c = 1) of op(B)_lj = x + iy;
// so that the real product of the two embedded operands is C with its real and imaginary parts in
// rows 2i and 2i + 1.  conj negates y (conjugate transposes).  The zero pattern (keep 1: l <= i,
// 2: l >= i; absolute l = local l + koff) refers to the complex indices.
struct Opnd {
  const void* X;
  long long sr, sk;
  int keep, cx, conj, koff;
};

__device__ __forceinline__ double opnd_at(const Opnd& o, long long r, long long k) {
  if (o.cx == 0) {
    if (!kept(o.keep, r, k + o.koff)) return 0.0;
    return static_cast<const double*>(o.X)[r * o.sr + k * o.sk];
  }
  const long long ri = (o.cx == 1) ? (r >> 1) : r, ki = k >> 1;
  if (!kept(o.keep, ri, ki + o.koff)) return 0.0;
  const double2 z = static_cast<const double2*>(o.X)[ri * o.sr + ki * o.sk];
  const double y = o.conj ? -z.y : z.y;
  if (o.cx == 2) return (k & 1) ? y : z.x;
  const long long a = r & 1, b = k & 1;
  return (a == b) ? z.x : (a == 0 ? -y : y);
}

// E[r] = max exponent over the kept entries of vector r (R vectors of K elements).  E holds a very
// negative value on entry (atomicMax).  Block 32 x 8; grid.y covers K in slices of 1024.
// fast_r: consecutive vectors are adjacent in memory (threads run across vectors); otherwise a
// warp reads along one vector.
__global__ void k_vec_exp(int R, int K, Opnd o, int fast_r, int* E) {
  const int k_lo = blockIdx.y * 1024, k_hi = min(K, k_lo + 1024);
  if (fast_r) {
    const int r = blockIdx.x * 32 + threadIdx.x;
    if (r >= R) return;
    int e = EXP_ZERO;
    for (int k = k_lo + threadIdx.y; k < k_hi; k += 8) e = max(e, exp_above(opnd_at(o, r, k)));
    if (e != EXP_ZERO) atomicMax(&E[r], e);
  } else {
    const int r = blockIdx.x * 8 + threadIdx.y;
    if (r >= R) return;  // uniform across the warp
    int e = EXP_ZERO;
    for (int k = k_lo + threadIdx.x; k < k_hi; k += 32) e = max(e, exp_above(opnd_at(o, r, k)));
    e = __reduce_max_sync(0xffffffffu, e);
    if (threadIdx.x == 0 && e != EXP_ZERO) atomicMax(&E[r], e);
  }
}

__device__ __forceinline__ int clamp_exp(int e) { return e < -1100 ? EXP_ZERO : e; }

// the balanced radix-2^7 digits of x 2^(55-E) (|x| < 2^E), as BF16 bit patterns of a_p 2^-7p
__device__ __forceinline__ void digits(double x, int E, uint16_t out[NSLICE]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF);
  long long X = 0;
  if (E < EXP_BAD && (be != 0 || (bits << 1) != 0)) {
    unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    int ex;
    if (be == 0) { ex = -1022; } else { m |= (1ull << 52); ex = be - 1023; }
    const int s = ex + 3 - E;  // X = m 2^(ex - 52 + 55 - E); s <= 2 since |x| < 2^E
    unsigned long long u = 0;
    if (s >= 0) u = m << s;
    else if (s > -64) u = m >> (-s);  // bits below 2^-55 of the scale are dropped
    X = (bits >> 63) ? -(long long)u : (long long)u;
  }
#pragma unroll
  for (int p = 1; p <= NSLICE; ++p) {
    const int sh = 56 - 7 * p;
    long long a;
    if (sh > 0) a = (X + (1ll << (sh - 1))) >> sh;  // nearest integer to X 2^-sh: |a| <= 64
    else a = X;
    X -= a * (1ll << sh);
    const float v = (float)a * __int_as_float((127 - 7 * p) << 23);  // a 2^-7p, exact
    out[p - 1] = __bfloat16_as_ushort(__float2bfloat16_rn(v));         // exact: |a| <= 64
  }
}

// Digit planes of one operand: vector r (a row of op(A) or a column of op(B)), element k, rows
// padded to RT tiles of TR, k to KT slices of 16.  One thread per (r, 8 consecutive k): it writes
// 16 bytes to each of the 8 planes of tile (r / TR, k / 16).
__global__ void k_split(int R, int K, Opnd o, int fast_r, const int* E, int TR, int RT, int KT, unsigned char* out) {
  const long long Rp = (long long)RT * TR, G = 2LL * KT;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= Rp * G) return;
  long long r, g;
  if (fast_r) { r = t % Rp; g = t / Rp; } else { g = t % G; r = t / G; }
  const int Er = (r < R) ? clamp_exp(E[r]) : EXP_ZERO;
  uint16_t dg[8][NSLICE];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const long long k = g * 8 + q;
    const double v = (r < R && k < K) ? opnd_at(o, r, k) : 0.0;
    digits(v, Er, dg[q]);
  }
  const long long rt = r / TR, kt = g >> 1;
  const int tile_bytes = TR * KS * 2;
  unsigned char* base =
      out + ((rt * KT + kt) * NSLICE) * (long long)tile_bytes + toff16((int)(r % TR), (int)(g & 1) * 8);
#pragma unroll
  for (int p = 0; p < NSLICE; ++p) {
    uint4 v;
    v.x = (uint32_t)dg[0][p] | ((uint32_t)dg[1][p] << 16);
    v.y = (uint32_t)dg[2][p] | ((uint32_t)dg[3][p] << 16);
    v.z = (uint32_t)dg[4][p] | ((uint32_t)dg[5][p] << 16);
    v.w = (uint32_t)dg[6][p] | ((uint32_t)dg[7][p] << 16);
    *reinterpret_cast<uint4*>(base + (long long)p * tile_bytes) = v;
  }
}

// K slices of a row tile of a block-diagonal op(A): the first slice of the tile's K range and the
// count (bm, bk multiples of 16 that divide / are multiples of the 128-row tile)
__host__ __device__ __forceinline__ void bd_range(int bm, int bk, int mt, int* first, int* count) {
  if (bm <= OM) {
    const int per = OM / bm;
    *first = mt * per * bk / KS;
    *count = per * bk / KS;
  } else {
    *first = (mt / (bm / OM)) * bk / KS;
    *count = bk / KS;
  }
}

// Entry (i, kk) (embedded units for complex data) of a block-diagonal back-transform-2 operand.
__device__ __forceinline__ double bd_at(const BdOp& o, long long i, long long kk) {
  const long long ir = o.cx ? (i >> 1) : i, kr = o.cx ? (kk >> 1) : kk;
  const int b = o.b;
  double x = 0.0, y = 0.0;
  if (o.kind == 1) {  // V_j^H: row q of block j, column r of the block's window
    const long long j = ir / b, q = ir % b, r = kr - 2LL * b * j;
    if (r < 0 || r >= 2 * b || j >= o.nblk) return 0.0;
    const long long g = o.g_lo + j, t = o.L - (o.ngroups - 1 - g), sw = g * b + q, rel = r - q;
    if (sw > o.n - 3 || rel < 0 || rel >= b || o.w00 + 2LL * b * j + r >= o.n) return 0.0;
    const long long rid = sw * o.ntask + t;
    if (o.cx) {
      const double2 tau = static_cast<const double2*>(o.tau2)[rid];
      if (tau.x == 0.0 && tau.y == 0.0) return 0.0;
      const double2 v = static_cast<const double2*>(o.V2)[rid * b + rel];
      x = v.x;
      y = -v.y;  // conjugate: op(A) = V^H
    } else {
      if (static_cast<const double*>(o.tau2)[rid] == 0.0) return 0.0;
      return static_cast<const double*>(o.V2)[rid * b + rel];
    }
  } else {  // W_j: row r of block j, column q
    const long long j = ir / (2 * b), r = ir % (2 * b), q = kr - (long long)b * j;
    if (q < 0 || q >= b || j >= o.nblk) return 0.0;
    const long long off = j * 2LL * b * b + r + q * 2LL * b;
    if (o.cx) {
      const double2 w = static_cast<const double2*>(o.W)[off];
      x = w.x;
      y = w.y;
    } else {
      return static_cast<const double*>(o.W)[off];
    }
  }
  const long long a = i & 1, c = kk & 1;  // the 2 x 2 block [[x, -y], [y, x]]
  return (a == c) ? x : (a == 0 ? -y : y);
}

// Row exponents and digit planes of a block-diagonal op(A) in the compact layout: row tile mt holds
// only the slices of its K range (bd_range).  One warp per row of the padded MT x 128 rows; lane l
// takes 8 consecutive columns of the range and writes 16 bytes to each plane.
__global__ void k_split_bd(int M, BdOp o, int bm, int bk, int MT, int* E, unsigned char* out) {
  const long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= (long long)MT * OM) return;  // uniform per warp
  const int mt = (int)(i / OM);
  int f = 0, c = 0;
  bd_range(bm, bk, mt, &f, &c);
  const bool act = lane * 8 < c * KS;
  double v[8];
  int e = EXP_ZERO;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const long long kk = (long long)f * KS + lane * 8 + q;
    v[q] = (act && i < M) ? bd_at(o, i, kk) : 0.0;
    e = max(e, exp_above(v[q]));
  }
  e = __reduce_max_sync(0xffffffffu, e);
  if (lane == 0) E[i] = e;
  if (!act) return;
  const int Er = clamp_exp(e);
  uint16_t dg[8][NSLICE];
#pragma unroll
  for (int q = 0; q < 8; ++q) digits(v[q], Er, dg[q]);
  const int tile_bytes = OM * KS * 2;
  unsigned char* base = out + (((long long)mt * c + (lane >> 1)) * NSLICE) * tile_bytes + toff16((int)(i % OM), (lane & 1) * 8);
#pragma unroll
  for (int p = 0; p < NSLICE; ++p) {
    uint4 w;
    w.x = (uint32_t)dg[0][p] | ((uint32_t)dg[1][p] << 16);
    w.y = (uint32_t)dg[2][p] | ((uint32_t)dg[3][p] << 16);
    w.z = (uint32_t)dg[4][p] | ((uint32_t)dg[5][p] << 16);
    w.w = (uint32_t)dg[6][p] | ((uint32_t)dg[7][p] << 16);
    *reinterpret_cast<uint4*>(base + (long long)p * tile_bytes) = w;
  }
}

struct OzP {
  int M, N, K, koff, c_lower, tri_a, tri_b, cx;  // cx: complex product in the real embedding
  int MT, NT, KT, ksplit;
  double alpha, beta;
  double* C;
  long long ldc;
  double* ws;  // split-K partials (ksplit > 1): ws[z M N + i + j M]
  const unsigned char* Ap;
  const unsigned char* Bp;
  const int* E;
  const int* F;
  int* status;
  // block-diagonal op(A) (0: off): block j has rows [j bd_bm, (j+1) bd_bm) and its non-zero columns
  // [j bd_bk, (j+1) bd_bk); the A planes then hold, per row tile, only that tile's K range (compact)
  int bd_bm, bd_bk;
};


// an exact FP32 chunk sum (a multiple of 2^-49 below 2^8 in magnitude) in units of 2^-49
__device__ __forceinline__ long long units49(uint32_t b) {
  const uint32_t e = (b >> 23) & 0xFF;
  const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u) << 40;
  unsigned long long t;
  asm("shr.b64 %0, %1, %2;" : "=l"(t) : "l"(m), "r"(141u - e));  // m 2^(e - 101); 0 for e = 0
  return (b >> 31) ? -(long long)t : (long long)t;
}

// x 2^e without a library call (two exact power-of-two factors cover |e| <= 2046)
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }
__device__ __forceinline__ double scale2(double x, int e) {
  if (e >= -1022 && e <= 1023) return x * pow2(e);
  e = max(-2044, min(2046, e));
  const int h = e / 2;
  return (x * pow2(h)) * pow2(e - h);
}


// (a 10-warp CTA puts 3 warps on one SM sub-partition of 16K registers: at most 168 registers per thread)
__global__ void __launch_bounds__(NTH, 1) ozaki_kernel(OzP p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // grouped raster: GROUP_M row tiles sweep the column tiles together
  const int per_group = GROUP_M * p.NT;
  const int first = (blockIdx.x / per_group) * GROUP_M;
  const int gm = min(p.MT - first, GROUP_M);
  const int within = blockIdx.x % per_group;
  const int mt = first + within % gm, nt = within / gm;
  const int m0 = mt * OM, n0 = nt * ON;
  // complex products: rows 2i, 2i + 1 and elements 2l, 2l + 1 belong to complex row i / element l
  const int rs = p.cx ? 1 : 0;
  const long long mr0 = m0 >> rs, mrn = OM >> rs;
  if (p.c_lower && n0 > mr0 + mrn - 1) return;
  // k-slices holding non-zero products for this tile (absolute k = local k + koff)
  long long kb = 0, ke = p.K >> rs;
  if (p.tri_a == 1) ke = std::min<long long>(ke, mr0 + mrn - p.koff);
  else if (p.tri_a == 2) kb = std::max<long long>(kb, mr0 - p.koff);
  if (p.tri_b == 1) kb = std::max<long long>(kb, (long long)n0 - p.koff);
  else if (p.tri_b == 2) ke = std::min<long long>(ke, (long long)n0 + ON - p.koff);
  kb <<= rs;
  ke <<= rs;
  int s_lo = (int)(kb / KS), s_hi = (int)(ke > 0 ? (ke + KS - 1) / KS : 0);
  if (s_hi < s_lo) s_hi = s_lo;
  // A-plane slices: a_kt per row tile, slice kt read at kt - a_off
  int a_kt = p.KT, a_off = 0;
  if (p.bd_bm) {
    int f = 0, c = 0;
    bd_range(p.bd_bm, p.bd_bk, mt, &f, &c);
    s_lo = min(f, p.KT);
    s_hi = min(f + c, p.KT);
    a_kt = c;
    a_off = f;
  }
  if (p.ksplit > 1) {  // this CTA's share of the slices
    const int tot = s_hi - s_lo, z = blockIdx.y;
    const int a = s_lo + (int)((long long)tot * z / p.ksplit);
    const int b = s_lo + (int)((long long)tot * (z + 1) / p.ksplit);
    s_lo = a;
    s_hi = b;
  }
  const int nst = s_hi - s_lo, nchunk = (nst + CHUNK - 1) / CHUNK;

  unsigned char* ctrl = smem + NSTAGE * STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(ctrl);  // [NSTAGE]: slice landed
  uint64_t* empty = full + NSTAGE;                      // [NSTAGE]: slice consumed by the MMAs
  uint64_t* cfull = empty + NSTAGE;                     // chunk accumulated
  uint64_t* cempty = cfull + 1;                         // chunk drained by the epilogue warps
  uint64_t* done = cempty + 1;                          // all MMAs complete
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ctrl + 256);
  volatile int* err = reinterpret_cast<volatile int*>(ctrl + 320);
  int* issued = reinterpret_cast<int*>(ctrl + 384);
  int* consumed = reinterpret_cast<int*>(ctrl + 448);
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(cfull)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(cempty)), "r"(NEPI_W));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(done)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *err = 0;
    *issued = 0;
    *consumed = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tslot)),
                 "r"(TMEM_COLS_OZ));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == NEPI_W) {
    // ---- copy warp: digit-plane slices into the stage ring
    if (lane == 0) {
      const unsigned char* a_src = p.Ap + ((long long)mt * a_kt - a_off) * A_STAGE;
      const unsigned char* b_src = p.Bp + (long long)nt * p.KT * B_STAGE;
      for (int s = 0; s < nst; ++s) {
        const int slot = s % NSTAGE;
        if (s >= NSTAGE && !bar_wait(su32(&empty[slot]), ((s / NSTAGE) - 1) & 1, err)) {
          if (!*err) *err = 411;
          break;
        }
        const uint32_t fb = su32(&full[slot]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(STAGE) : "memory");
        const uint32_t dst = su32(smem + slot * STAGE);
        const long long kt = s_lo + s;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
            "l"(a_src + kt * A_STAGE), "r"(A_STAGE), "r"(fb)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                dst + A_STAGE),
            "l"(b_src + kt * B_STAGE), "r"(B_STAGE), "r"(fb)
            : "memory");
        *issued = s + 1;
      }
    }
  } else if (warp == NEPI_W + 1) {
    // ---- MMA warp: 36 digit-pair products per 16-deep slice
    if (lane == 0) {
      const uint32_t id = idesc_bf16(OM, ON);
      for (int s = 0; s < nst; ++s) {
        const int slot = s % NSTAGE, c = s / CHUNK;
        const bool chunk_start = (s % CHUNK) == 0;
        if (chunk_start && c > 0 && !bar_wait(su32(cempty), (c - 1) & 1, err)) {
          if (!*err) *err = 412;
          break;
        }
        if (!bar_wait(su32(&full[slot]), (s / NSTAGE) & 1, err)) {
          if (!*err) *err = 413;
          break;
        }
        *consumed = s + 1;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t a0 = su32(smem + slot * STAGE), b0 = a0 + A_STAGE;
#pragma unroll
        for (int pa = 1; pa <= NSLICE; ++pa) {
#pragma unroll
          for (int qb = 1; qb + pa <= DMAX; ++qb) {
            const int d = pa + qb;
            int col, en;
            if (d <= DEXACT) {  // the first pair of diagonal d (pa = 1) restarts it at a chunk start
              col = (d - 2) * ON;
              en = (chunk_start && pa == 1) ? 0 : 1;
            } else {  // the shared slot starts with the first MMA of d = 8 (pa = 1, qb = 7)
              col = SHARED_SLOT * ON;
              en = (s == 0 && pa == 1 && qb == DEXACT) ? 0 : 1;
            }
            mma_bf16(tmem + col, sdesc16(a0 + (pa - 1) * A_TILE), sdesc16(b0 + (qb - 1) * B_TILE), id, en);
          }
        }
        commit(su32(&empty[slot]));
        if ((s % CHUNK) == CHUNK - 1 || s == nst - 1) commit(su32(cfull));
      }
      commit(su32(done));
      if (!bar_wait_plain(su32(done), 0) && !*err) *err = 414;
    }
  } else {
    // ---- epilogue warps: drain the exact diagonals per chunk, then write C
    const int quarter = warp & 3, col0 = (warp >> 2) * HC;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
    long long acc[HC];
#pragma unroll
    for (int c = 0; c < HC; ++c) acc[c] = 0;
    bool good = true;
    for (int c = 0; c < nchunk; ++c) {
      if (!bar_wait(su32(cfull), c & 1, err)) {
        if (!*err) *err = 415;
        good = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int d = 2; d <= DEXACT; ++d) {
        uint32_t r0[16], r1[16];
        tmem_ld16(lane_base + (uint32_t)((d - 2) * ON), r0);
        tmem_ld16(lane_base + (uint32_t)((d - 2) * ON + 16), r1);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          acc[q] += units49(r0[q]);
          acc[16 + q] += units49(r1[q]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(cempty)) : "memory");
    }
    const bool any = good && nchunk > 0;
    const int gi = m0 + row;
    const int Ei = (any && gi < p.M) ? p.E[gi] : EXP_ZERO;
#pragma unroll
    for (int cb = 0; cb < HC; cb += 16) {
      uint32_t r[16];
      if (any) {
        tmem_ld16(lane_base + (uint32_t)(SHARED_SLOT * ON + cb), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = 0u;
      }
      if (gi < p.M) {
#pragma unroll
        for (int h = 0; h < 16; h += 8) {
          // the loads of 8 outputs (column exponents, C) first, so that they overlap
          const bool read_c = p.ksplit == 1 && p.beta != 0.0;
          double cin[8];
          int fj[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int gj = n0 + col0 + cb + h + u;
            const bool ok = gj < p.N && !(p.c_lower && (gi >> rs) < gj);
            fj[u] = (ok && any) ? p.F[gj] : EXP_ZERO;
            cin[u] = (ok && read_c) ? p.C[gi + gj * p.ldc] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int q = h + u;
            const int gj = n0 + col0 + cb + q;
            if (gj >= p.N || (p.c_lower && (gi >> rs) < gj)) continue;
            double v = 0.0;
            if (any) {
              const int Fj = fj[u];
              if (Ei >= EXP_BAD || Fj >= EXP_BAD) {
                v = __longlong_as_double(0x7FF8000000000000ll);  // an Inf / NaN entry reached this output
              } else if (Ei >= -1100 && Fj >= -1100) {
                const double sum = (double)acc[cb + q] * 0x1p-49 + (double)__uint_as_float(r[q]);
                v = scale2(sum, Ei + Fj + 2);
              }
            }
            if (p.ksplit > 1) {
              p.ws[(long long)blockIdx.y * p.M * p.N + gi + (long long)gj * p.M] = v;
            } else {
              const double o = p.alpha * v;
              p.C[gi + gj * p.ldc] = read_c ? o + p.beta * cin[u] : o;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0 && *err) {
    // a wait gave up: let the copies already issued land before the shared memory is released
    for (int s = *consumed; s < *issued; ++s) bar_wait_plain(su32(&full[s % NSTAGE]), (s / NSTAGE) & 1);
    atomicCAS(&p.status[ST_TIMEOUT], 0, *err);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS_OZ));
}

// C = alpha sum_z ws[z] + beta C in a fixed order (deterministic)
// (rs = 1: complex product in the real embedding, rows 2i, 2i + 1 belong to complex row i)
__global__ void k_oz_reduce(int M, int N, int ks, int c_lower, int rs, double alpha, const double* ws, double beta,
                            double* C, long long ldc) {
  const long long total = (long long)M * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % M), j = (int)(t / M);
    if (c_lower && (i >> rs) < j) continue;
    double s = 0.0;
    for (int z = 0; z < ks; ++z) s += ws[(long long)z * total + t];
    double* c = &C[i + (long long)j * ldc];
    const double o = alpha * s;
    *c = (beta != 0.0) ? o + beta * (*c) : o;
  }
}

size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct OzLayout {
  size_t Mp, Np, Kp, f_off, a_off, b_off, total;
};

OzLayout oz_layout(int M, int N, int K) {
  OzLayout L;
  L.Mp = rup(std::max(M, 1), OM);
  L.Np = rup(std::max(N, 1), ON);
  L.Kp = rup(std::max(std::min(K, KMAX), 1), KS);
  L.f_off = rup(L.Mp * sizeof(int), 256);
  L.a_off = L.f_off + rup(L.Np * sizeof(int), 256);
  L.b_off = L.a_off + L.Mp * L.Kp * 2 * NSLICE;
  L.total = L.b_off + L.Np * L.Kp * 2 * NSLICE;
  return L;
}

}  // namespace

size_t gemm_f64_emulated_scratch(int M, int N, int K) { return oz_layout(M, N, K).total; }

namespace {

// C (M x N, real, ldc) = alpha op(A) op(B) + beta C with op(A) = the M x K operand a and op(B) the
// N x K operand b (vectors = columns of op(B)), K in the operands' element units (embedded for
// complex data); ka / kb: bytes of one underlying element step along K of a / b, to offset the
// K pieces of one launch; rs = 1 for complex products.
void emulate(Sys& s, int M, int N, int K, Opnd a, size_t a_kstep, Opnd b, size_t b_kstep, int tri_a, int tri_b,
             int c_lower, int rs, double alpha, double beta, double* C, long long ldc) {
  const OzLayout L = oz_layout(M, N, K);
  int site = 0;
  if (s.ozws == nullptr || L.total > s.ozws_bytes) {  // internal sizing error: fail the call loudly
    fprintf(stderr, "gev: emulated FP64 GEMM scratch too small (%zu < %zu bytes)\n", s.ozws_bytes, L.total);
    site = 499;
  } else if (allow_dyn_smem(ozaki_kernel, SMEM_OZ) != 0) {
    site = 498;
  }
  if (site) {  // recorded in the status words: the caller's next status check returns GEV_ERR_CUDA
    if (s.status) cudaMemcpyAsync(s.status + ST_CONFIG, &site, sizeof(int), cudaMemcpyHostToDevice, s.stream);
    cudaStreamSynchronize(s.stream);
    return;
  }
  unsigned char* base = static_cast<unsigned char*>(s.ozws);
  int* E = reinterpret_cast<int*>(base);
  int* F = reinterpret_cast<int*>(base + L.f_off);
  unsigned char* Ap = base + L.a_off;
  unsigned char* Bp = base + L.b_off;
  const int fast_a = a.sr == 1, fast_b = b.sr == 1;
  const int MT = (int)(L.Mp / OM), NT = (int)(L.Np / ON);
  for (int k0 = 0; k0 < std::max(K, 1); k0 += KMAX) {  // K pieces (k0 even: whole complex elements)
    const int Kc = std::max(0, std::min(KMAX, K - k0));
    const int KT = (Kc + KS - 1) / KS;
    const int ku = k0 >> rs;  // the piece's first underlying element along K
    Opnd ap = a, bp = b;
    ap.X = static_cast<const unsigned char*>(a.X) + (size_t)ku * a_kstep;
    bp.X = static_cast<const unsigned char*>(b.X) + (size_t)ku * b_kstep;
    ap.koff = bp.koff = ku;
    if (Kc > 0) {
      cudaMemsetAsync(E, 0x80, L.Mp * sizeof(int), s.stream);
      cudaMemsetAsync(F, 0x80, L.Np * sizeof(int), s.stream);
      const dim3 eb(32, 8);
      GEV_COUNT(s);
      k_vec_exp<<<dim3(fast_a ? cdiv(M, 32) : cdiv(M, 8), cdiv(Kc, 1024)), eb, 0, s.stream>>>(M, Kc, ap, fast_a, E);
      GEV_COUNT(s);
      k_vec_exp<<<dim3(fast_b ? cdiv(N, 32) : cdiv(N, 8), cdiv(Kc, 1024)), eb, 0, s.stream>>>(N, Kc, bp, fast_b, F);
      GEV_COUNT(s);
      k_split<<<cdiv((long long)MT * OM * 2 * KT, 256), 256, 0, s.stream>>>(M, Kc, ap, fast_a, E, OM, MT, KT, Ap);
      GEV_COUNT(s);
      k_split<<<cdiv((long long)NT * ON * 2 * KT, 256), 256, 0, s.stream>>>(N, Kc, bp, fast_b, F, ON, NT, KT, Bp);
    }
    OzP p{};
    p.M = M; p.N = N; p.K = Kc; p.koff = ku; p.c_lower = c_lower;
    p.tri_a = tri_a; p.tri_b = tri_b; p.cx = rs;
    p.MT = MT; p.NT = NT; p.KT = KT;
    p.alpha = alpha; p.beta = (k0 == 0) ? beta : 1.0;
    p.C = C; p.ldc = ldc; p.Ap = Ap; p.Bp = Bp; p.E = E; p.F = F; p.status = s.status;
    // split K when the output has too few tiles to fill the GPU and K is long
    long long tiles = (long long)MT * NT;
    if (c_lower) tiles = (tiles + MT) / 2;
    int ks = 1;
    if (tiles < s.sms && KT >= 2 * CHUNK) {
      ks = (int)std::min<long long>((2LL * s.sms + tiles - 1) / tiles, KT / CHUNK);
      ks = std::min(ks, 16);
      while (ks > 1 && (size_t)ks * M * N * sizeof(double) > s.splitws_bytes) --ks;
    }
    p.ksplit = ks;
    p.ws = ks > 1 ? static_cast<double*>(s.splitws) : nullptr;
    GEV_COUNT(s);
    ozaki_kernel<<<dim3(MT * NT, ks), NTH, SMEM_OZ, s.stream>>>(p);
    if (ks > 1) {
      const long long total = (long long)M * N;
      unsigned blocks = cdiv(total, 256);
      if (blocks > 8u * s.sms) blocks = 8u * s.sms;
      GEV_COUNT(s);
      k_oz_reduce<<<blocks, 256, 0, s.stream>>>(M, N, ks, c_lower, rs, p.alpha, p.ws, p.beta, C, ldc);
    }
  }
}

int keep_a_of(int tri_a) { return tri_a == 1 ? 1 : (tri_a == 2 ? 2 : 0); }
int keep_b_of(int tri_b) { return tri_b == 1 ? 2 : (tri_b == 2 ? 1 : 0); }

}  // namespace

// FP64 GEMM on the tensor cores (real data); scratch s.ozws of s.ozws_bytes >= gemm_f64_emulated_scratch.
// Zero patterns: op(A)[i,k] = 0 for k > i (tri_a 1) or k < i (tri_a 2); op(B)[k,j] = 0 for k < j
// (tri_b 1) or k > j (tri_b 2).
void gemm_f64_emulated(Sys& s, const GemmP<double>& q) {
  if (q.M <= 0 || q.N <= 0) return;
  // op(A) row i, element k: A[i + k lda] (ta 0) or A[k + i lda]; op(B) column j, element k:
  // B[k + j ldb] (tb 0) or B[j + k ldb]
  Opnd a{q.A, q.ta ? q.lda : 1, q.ta ? 1 : q.lda, keep_a_of(q.tri_a), 0, 0, 0};
  Opnd b{q.B, q.tb ? 1 : q.ldb, q.tb ? q.ldb : 1, keep_b_of(q.tri_b), 0, 0, 0};
  emulate(s, q.M, q.N, q.K, a, sizeof(double) * (size_t)a.sk, b, sizeof(double) * (size_t)b.sk, q.tri_a, q.tri_b,
          q.c_lower, 0, q.alpha, q.beta, q.C, q.ldc);
}

// Complex FP64 GEMM on the tensor cores through the real embedding (2M x 2K) (2K x N): the
// result's real and imaginary parts are rows 2i and 2i + 1 of the real view of C (leading
// dimension 2 ldc).  alpha and beta must be real (the caller checks).  ta / tb 2: conjugate
// transposes.
void gemm_c128_emulated(Sys& s, const GemmP<zd>& q) {
  if (q.M <= 0 || q.N <= 0) return;
  Opnd a{q.A, q.ta ? q.lda : 1, q.ta ? 1 : q.lda, keep_a_of(q.tri_a), 1, q.ta == 2 ? 1 : 0, 0};
  Opnd b{q.B, q.tb ? 1 : q.ldb, q.tb ? q.ldb : 1, keep_b_of(q.tri_b), 2, q.tb == 2 ? 1 : 0, 0};
  emulate(s, 2 * q.M, q.N, 2 * q.K, a, sizeof(zd) * (size_t)a.sk, b, sizeof(zd) * (size_t)b.sk, q.tri_a, q.tri_b,
          q.c_lower, 1, q.alpha.x, q.beta.x, reinterpret_cast<double*>(q.C), 2 * q.ldc);
}

namespace {

struct BdLayout {
  size_t Mp, Np, f_off, a_off, b_off, total;
  int MT, NT, KT, acount;
};

// scratch of a block-diagonal product (embedded units): row exponents, column exponents, the compact
// A planes (acount slices per row tile) and the B planes over the whole K (no piece limit: a tile
// sums at most 16 slices, far below the int64 accumulator's range)
BdLayout bd_layout(int Me, int N, int Ke, int bme, int bke) {
  BdLayout L;
  L.Mp = rup(std::max(Me, 1), OM);
  L.Np = rup(std::max(N, 1), ON);
  L.MT = (int)(L.Mp / OM);
  L.NT = (int)(L.Np / ON);
  L.KT = (std::max(Ke, 1) + KS - 1) / KS;
  int f = 0;
  bd_range(bme, bke, 0, &f, &L.acount);
  L.f_off = rup(L.Mp * sizeof(int), 256);
  L.a_off = L.f_off + rup(L.Np * sizeof(int), 256);
  L.b_off = L.a_off + (size_t)L.MT * L.acount * A_STAGE;
  L.total = L.b_off + (size_t)L.NT * L.KT * B_STAGE;
  return L;
}

}  // namespace

size_t gemm_f64_bdiag_scratch(int M, int N, int K, int bm, int bk, int cx) {
  const int e = cx ? 2 : 1;
  return bd_layout(e * M, N, e * K, e * bm, e * bk).total;
}

namespace {
__global__ void k_fill_exp(int n, int v, int* E) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) E[i] = v;
}
}  // namespace

bool gemm_f64_bdiag(Sys& s, int M, int N, int K, const BdOp& a, int bm, int bk, const void* B, long long ldb,
                    double alpha, double beta, void* C, long long ldc, bool b_below_two) {
  if (M <= 0 || N <= 0) return true;
  const int rs = a.cx ? 1 : 0;
  const int Me = M << rs, Ke = K << rs, bme = bm << rs, bke = bk << rs;
  const BdLayout L = bd_layout(Me, N, Ke, bme, bke);
  if (!s.ozws || L.total > s.ozws_bytes) return false;
  if (allow_dyn_smem(ozaki_kernel, SMEM_OZ) != 0) return false;
  unsigned char* base = static_cast<unsigned char*>(s.ozws);
  int* E = reinterpret_cast<int*>(base);
  int* F = reinterpret_cast<int*>(base + L.f_off);
  unsigned char* Ap = base + L.a_off;
  unsigned char* Bp = base + L.b_off;
  // op(B) column j, element k: B[k + j ldb] (complex: the re / im parts of element k / 2)
  const Opnd b{B, ldb, 1, 0, a.cx ? 2 : 0, 0, 0};
  GEV_COUNT(s);
  k_split_bd<<<cdiv((long long)L.MT * OM * 32, 256), 256, 0, s.stream>>>(Me, a, bme, bke, L.MT, E, Ap);
  if (b_below_two) {  // every entry of B below 2 in magnitude: the column exponents are 1, no pass over B
    GEV_COUNT(s);
    k_fill_exp<<<cdiv(L.Np, 256), 256, 0, s.stream>>>((int)L.Np, 1, F);
  } else {
    cudaMemsetAsync(F, 0x80, L.Np * sizeof(int), s.stream);
  }
  if (Ke > 0) {
    if (!b_below_two) {
      GEV_COUNT(s);
      k_vec_exp<<<dim3(cdiv(N, 8), cdiv(Ke, 1024)), dim3(32, 8), 0, s.stream>>>(N, Ke, b, 0, F);
    }
    GEV_COUNT(s);
    k_split<<<cdiv((long long)L.NT * ON * 2 * L.KT, 256), 256, 0, s.stream>>>(N, Ke, b, 0, F, ON, L.NT, L.KT, Bp);
  }
  OzP p{};
  p.M = Me; p.N = N; p.K = Ke; p.koff = 0; p.c_lower = 0;
  p.tri_a = 0; p.tri_b = 0; p.cx = rs;
  p.MT = L.MT; p.NT = L.NT; p.KT = L.KT; p.ksplit = 1;
  p.alpha = alpha; p.beta = beta;
  p.C = static_cast<double*>(C);
  p.ldc = ldc << rs;
  p.ws = nullptr;
  p.Ap = Ap; p.Bp = Bp; p.E = E; p.F = F; p.status = s.status;
  p.bd_bm = bme;
  p.bd_bk = bke;
  GEV_COUNT(s);
  ozaki_kernel<<<dim3(L.MT * L.NT, 1), NTH, SMEM_OZ, s.stream>>>(p);
  return true;
}

}  // namespace gev

extern "C" size_t gev_gemm_f64_scratch_bytes(int M, int N, int K) {
  if (M < 0 || N < 0 || K < 0) return 0;
  return ((gev::gemm_f64_emulated_scratch(M, N, K) + 255) & ~(size_t)255) + ((size_t)16 << 20);
}

extern "C" int gev_gemm_f64(int M, int N, int K, int ta, int tb, double alpha, const double* A, int lda,
                            const double* B, int ldb, double beta, double* C, int ldc, int engine, void* stream,
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
  if (engine < 0 || engine > 1) return -14;
  if (!status_dev) return -16;
  if (engine == 1 && (!scratch_dev || scratch_bytes < gev_gemm_f64_scratch_bytes(M, N, K))) return -17;
  Sys s;
  s.stream = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  GEV_CUDA_TRY(cudaGetDevice(&dev));
  GEV_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  s.sms = sms > 0 ? sms : 152;
  s.status = status_dev;
  s.emu_fp64 = engine;
  if (engine == 1) {  // planes first, then the split-K partials
    const size_t planes = (gemm_f64_emulated_scratch(M, N, K) + 255) & ~(size_t)255;
    s.ozws = scratch_dev;
    s.ozws_bytes = planes;
    s.splitws = static_cast<unsigned char*>(scratch_dev) + planes;
    s.splitws_bytes = scratch_bytes - planes;
  } else {
    s.splitws = nullptr;
    s.splitws_bytes = 0;
  }
  gemm<double>(s, gp<double>(M, N, K, ta, tb, alpha, A, lda, B, ldb, beta, C, ldc));
  GEV_TRY(last_error());
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  return 0;
}
