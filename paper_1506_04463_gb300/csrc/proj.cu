// Tall-skinny projections of the Rayleigh-Ritz step on the tensor cores,
// FP64-accurate (Fig. alg:three steps 2.a and 4.a: B_Q = Q^H B Q,
// A_U = Uh^H A U, B_U = Uh^H B U):   G = X^H Y,  X: n x mx,  Y: n x my.
//
// The FP64 operands are cut into integer digits that BF16 holds exactly, the
// digit products are summed exactly on the tensor cores, and the levels are
// combined in 64-bit integers (an error-free splitting in the spirit of
// Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012; here with fixed-point digits):
//
//  * every column c of X (and of Y) gets the exponent field F_c of its
//    largest |Re|, |Im| (so that |v| < 2^(F_c - 1022) for all its entries);
//  * a value v of column c is the 55-bit fixed-point integer
//    J = trunc(v 2^(1077 - F_c)), |J| < 2^55, written in eight balanced
//    base-128 digits J = sum_s d_s 2^(7(7-s)), |d_s| <= 64 (s = 0..7);
//  * a product is x y = 2^(F_x + F_y - 2154) sum_{s,t} d_s e_t 2^(7(14-s-t));
//    the 36 digit pairs with s + t <= 7 are kept (level g = s + t); the
//    dropped pairs weigh below 2^-53 of max|x| max|y|;
//  * the complex product conj(x) y is a real dot product over interleaved
//    (Re, Im) pairs: GEMM row a of A' is (Re x_a, Im x_a), row 64 + a is
//    (-Im x_a, Re x_a), row b of B' is (Re y_b, Im y_b), so that rows a and
//    64 + a of D = A' B'^T give Re G and Im G.
//
// k_gram_tc: a CTA takes a 64 x 64 block of G and a chunk of rows.  Per
// stage of 16 rows (32 real K), 512 threads write the digit planes of A'
// (128 x 32) and B' (64 x 32) as BF16 into shared memory (double-buffered),
// and one thread issues the 36 x 2 tcgen05.mma (M = 128, N = 64, K = 16) of
// the stage into eight FP32 accumulators in tensor memory, one per level.
// Every 4 stages the levels (each |sum| <= 8 * 64 * 64 * 128 = 2^22, so FP32
// holds it exactly) are read with tcgen05.ld and folded into two exact int64
// accumulators per element: hi = sum_{g<=3} acc_g 2^(7(3-g)),
// lo = sum_{g>=4} acc_g 2^(7(7-g)), value = 2^(F_x+F_y-2105) (hi 2^28 + lo).
// Per-CTA partials are summed exactly in int64 by k_gram_tc_reduce, which
// rounds once to FP64.  The result does not depend on the chunking.
#include <algorithm>
#include <atomic>
#include "kernels.h"
#include "tc.cuh"

namespace {

constexpr int kS = 8;                         // digits per value
constexpr int kKS = 32;                       // real K per stage
constexpr int kRows = kKS / 2;                // complex rows per stage
constexpr int kFlush = 4;                     // stages per flush (128 real K)
constexpr int kMA = 128;                      // A' rows: 64 columns of X, two forms
constexpr int kNB = 64;                       // B' rows: 64 columns of Y
constexpr int kCoreK = 128;                   // LBO: bytes between core matrices along K
constexpr int kSBO = (kKS / 8) * 128;         // bytes between 8-row groups: 512
constexpr int kAPlane = kMA * kKS * 2;        // 8192 bytes
constexpr int kBPlane = kNB * kKS * 2;        // 4096 bytes
constexpr int kBuf = kS * (kAPlane + kBPlane);  // 98304 bytes per stage buffer
constexpr int kThreads = 512;
constexpr uint32_t kIdescG = tc::idesc_bf16(kMA, kNB);
constexpr int kTmemCols = 512;                // 8 levels x 64 columns

__device__ __forceinline__ int canon(int row, int k) {
  return (row >> 3) * kSBO + (k >> 3) * kCoreK + (row & 7) * 16 + (k & 7) * 2;
}

// exponent field of |v| (0 for zero and subnormals)
__device__ __forceinline__ int expo_field(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7FF);
}

// Balanced base-128 digits of the 55-bit fixed-point image of v in a column
// with exponent field F (see the file comment); d[0] is the leading digit.
__device__ __forceinline__ void split_digits(double v, int F, int (&d)[kS]) {
  const long long bits = __double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7FF);
  long long J = 0;
  if (e != 0) {
    const long long mant = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const int sh = e - F + 2;  // <= 2 because e <= F
    J = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ll);
    if (bits < 0) J = -J;
  }
  // low part: 28 bits as four digits, in 32-bit arithmetic; the carry goes up
  int lo = (int)(J & 0xFFFFFFF);
  long long hi = J >> 28;
#pragma unroll
  for (int s = kS - 1; s >= 4; --s) {
    const int dd = ((lo + 64) & 127) - 64;
    d[s] = dd;
    lo = (lo - dd) >> 7;
  }
  int h = (int)hi + lo;  // |h| < 2^27 + 1
#pragma unroll
  for (int s = 3; s >= 1; --s) {
    const int dd = ((h + 64) & 127) - 64;
    d[s] = dd;
    h = (h - dd) >> 7;
  }
  d[0] = h;
}

// two small integers (|x| < 2^22) as a packed BF16 pair (lo in the low half)
__device__ __forceinline__ uint32_t bf16_pair(int lo, int hi) {
  const float flo = __int_as_float(0x4B400000 + lo) - 12582912.f;
  const float fhi = __int_as_float(0x4B400000 + hi) - 12582912.f;
  return __byte_perm(__float_as_uint(flo), __float_as_uint(fhi), 0x7632);
}

// FP32 holding an integer of modulus <= 2^22 -> that integer
__device__ __forceinline__ int f2i_exact(float v) { return __float_as_int(v + 12582912.f) - 0x4B400000; }

// (hi 2^28 + lo) 2^E rounded once to FP64 (round half away from zero), in
// integer arithmetic; results below the normal range flush to zero.
__device__ __forceinline__ double fix_to_double(long long hi, long long lo, int E) {
  const __int128 T = ((__int128)hi << 28) + (__int128)lo;
  if (T == 0) return 0.0;
  const bool neg = T < 0;
  const unsigned __int128 U = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
  const unsigned long long uh = (unsigned long long)(U >> 64), ul = (unsigned long long)U;
  const int p = uh ? 127 - __clzll((long long)uh) : 63 - __clzll((long long)ul);  // leading bit
  unsigned long long m = p >= 53 ? (unsigned long long)(U >> (p - 53)) : (unsigned long long)U << (53 - p);
  m = (m + 1) >> 1;  // 53 significant bits, rounded
  int ex = p + E;
  if (m >> 53) {
    m >>= 1;
    ++ex;
  }
  const int biased = ex + 1023;
  if (biased <= 0) return neg ? -0.0 : 0.0;
  if (biased >= 2047) return neg ? -__longlong_as_double(0x7FF0000000000000ll) : __longlong_as_double(0x7FF0000000000000ll);
  return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)biased << 52) |
                                          (m & ((1ull << 52) - 1))));
}

}  // namespace

// Column exponent fields: F[c] = max over the rows of the exponent field of
// |Re X[r][c]| and |Im X[r][c]| (F must be zeroed before).  blockIdx.y picks
// X (0) or Y (1).
__global__ void __launch_bounds__(256) k_col_expo(const cxd *__restrict__ X, int ldx, int mx, const cxd *__restrict__ Y,
                                                  int ldy, int my, int n, int rows_per_cta, int *FX, int *FY) {
  __shared__ int sm[kMaxM0];
  const cxd *M = blockIdx.y ? Y : X;
  const int ld = blockIdx.y ? ldy : ldx, m = blockIdx.y ? my : mx;
  int *F = blockIdx.y ? FY : FX;
  for (int c = threadIdx.x; c < m; c += blockDim.x) sm[c] = 0;
  __syncthreads();
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  const long long cnt = r1 > r0 ? (long long)(r1 - r0) * m : 0;
  int cur = -1, em = 0;
  for (long long idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
    const int r = (int)(idx / m), c = (int)(idx - (long long)r * m);
    if (c != cur) {
      if (cur >= 0) atomicMax(&sm[cur], em);
      cur = c;
      em = 0;
    }
    const cxd v = M[(size_t)(r0 + r) * ld + c];
    em = max(em, max(expo_field(v.re), expo_field(v.im)));
  }
  if (cur >= 0) atomicMax(&sm[cur], em);
  __syncthreads();
  for (int c = threadIdx.x; c < m; c += blockDim.x)
    if (sm[c]) atomicMax(&F[c], sm[c]);
}

__global__ void __launch_bounds__(kThreads, 1) k_gram_tc(const cxd *__restrict__ X, int ldx, int mx,
                                                         const cxd *__restrict__ Y, int ldy, int my, int n,
                                                         int rows_per_cta, const int *__restrict__ FX,
                                                         const int *__restrict__ FY, long long *__restrict__ part,
                                                         int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * kBuf);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 2 * kBuf + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int a0 = blockIdx.y * 64, b0 = blockIdx.z * 64;
  const int rb = blockIdx.x * rows_per_cta, re = min(n, rb + rows_per_cta);
  const int nst = re > rb ? (re - rb + kRows - 1) / kRows : 0;

  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
  }
  if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
  tc::fence_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;

  // this thread's conversion items: 4 per stage (2 of X, 2 of Y); lanes of a
  // warp cover 8 consecutive columns x 4 consecutive rows (conflict-free
  // 4-byte stores into the canonical layout, 128-byte global segments)
  auto convert = [&](int st, int buf) {
    unsigned char *Ab = smem + buf * kBuf;
    unsigned char *Bb = Ab + kS * kAPlane;
    const int r0 = rb + st * kRows;
    cxd v[4];
    int F[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = (tid + j * kThreads) & 1023;
      const int w = e >> 5, ln = e & 31;
      const int col = (w & 7) * 8 + (ln & 7), r = (w >> 3) * 4 + (ln >> 3);
      const int row = r0 + r;
      const bool isY = j >= 2;
      const int c = (isY ? b0 : a0) + col;
      const bool ok = row < re && c < (isY ? my : mx);
      v[j] = ok ? (isY ? Y[(size_t)row * ldy + c] : X[(size_t)row * ldx + c]) : mk(0.0, 0.0);
      F[j] = ok ? (isY ? FY[c] : FX[c]) : 0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = (tid + j * kThreads) & 1023;
      const int w = e >> 5, ln = e & 31;
      const int col = (w & 7) * 8 + (ln & 7), r = (w >> 3) * 4 + (ln >> 3);
      int dr[kS], di[kS];
      split_digits(v[j].re, F[j], dr);
      split_digits(v[j].im, F[j], di);
      if (j < 2) {
        const int o1 = canon(col, 2 * r), o2 = canon(64 + col, 2 * r);
#pragma unroll
        for (int s = 0; s < kS; ++s) {
          *reinterpret_cast<uint32_t *>(Ab + s * kAPlane + o1) = bf16_pair(dr[s], di[s]);
          *reinterpret_cast<uint32_t *>(Ab + s * kAPlane + o2) = bf16_pair(-di[s], dr[s]);
        }
      } else {
        const int o = canon(col, 2 * r);
#pragma unroll
        for (int s = 0; s < kS; ++s) *reinterpret_cast<uint32_t *>(Bb + s * kBPlane + o) = bf16_pair(dr[s], di[s]);
      }
    }
  };

  long long hi[16], lo[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
  const int q = warp & 3, cg = warp >> 2;  // TMEM lane quarter, 16-column group

  if (nst > 0) convert(0, 0);
  tc::fence_smem();
  __syncthreads();
  bool ok = true;
  int issued = 0;
  for (int st = 0; st < nst; ++st) {
    const int b = st & 1;
    if (tid == 0) {
      tc::fence_after();
      const uint32_t abase = tc::smem_u32(smem + b * kBuf), bbase = abase + kS * kAPlane;
      const bool first = (st % kFlush) == 0;
#pragma unroll
      for (int g = 0; g < kS; ++g)
#pragma unroll
        for (int s = 0; s <= g; ++s)
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            tc::mma(tmem + 64 * g, tc::smem_desc(abase + s * kAPlane + kk * 2 * kCoreK, kCoreK, kSBO),
                    tc::smem_desc(bbase + (g - s) * kBPlane + kk * 2 * kCoreK, kCoreK, kSBO), kIdescG,
                    (first && s == 0 && kk == 0) ? 0u : 1u);
      tc::commit(&bar[b]);
    }
    issued = st + 1;
    if (st + 1 < nst) {
      // the other buffer is free once the previous stage's products are done
      const bool w1 = st >= 1 ? tc::mbar_wait(&bar[b ^ 1], ((st - 1) >> 1) & 1) : true;
      if (__syncthreads_or(!w1)) {
        ok = false;
        break;
      }
      convert(st + 1, b ^ 1);
      tc::fence_smem();
    }
    if (st % kFlush == kFlush - 1 || st == nst - 1) {
      const bool w2 = tc::mbar_wait(&bar[b], (st >> 1) & 1);
      if (__syncthreads_or(!w2)) {
        ok = false;
        break;
      }
      tc::fence_after();
#pragma unroll
      for (int g = 0; g < kS; ++g) {
        float v[16];
        tc::ld16(tmem + ((uint32_t)(q * 32) << 16) + 64 * g + 16 * cg, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const long long iv = f2i_exact(v[c]);
          if (g <= 3)
            hi[c] += iv << (7 * (3 - g));
          else
            lo[c] += iv << (7 * (7 - g));
        }
      }
      tc::fence_before();
    }
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) {
      atomicOr(err, DEVERR_TIMEOUT);
      // bounded wait for the products still in flight before freeing TMEM
      if (issued >= 1) tc::mbar_wait(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
    }
  } else {
    const int tile = blockIdx.y * gridDim.z + blockIdx.z;
    const int row = q * 32 + lane;
    longlong2 *dst = reinterpret_cast<longlong2 *>(
        part + ((((size_t)tile * gridDim.x + blockIdx.x) * kMA + row) * kNB + 16 * cg) * 2);
#pragma unroll
    for (int c = 0; c < 16; ++c) dst[c] = make_longlong2(hi[c], lo[c]);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_free(tmem, kTmemCols);
}

// G[a][b] from the partials of k_gram_tc: exact int64 sums over the chunks,
// scaled by 2^(F_a + F_b - 2105) and rounded once to FP64.  Thread (row, col)
// of tile (blockIdx.y, blockIdx.z): row < 64 -> Re G, row >= 64 -> Im G.
__global__ void __launch_bounds__(256) k_gram_tc_reduce(const long long *__restrict__ part, int nchunks, int mx,
                                                        int my, const int *__restrict__ FX,
                                                        const int *__restrict__ FY, cxd *__restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kMA * kNB) return;
  const int row = e / kNB, col = e - row * kNB;
  const int a = blockIdx.y * 64 + (row & 63), b = blockIdx.z * 64 + col;
  if (a >= mx || b >= my) return;
  const int tile = blockIdx.y * gridDim.z + blockIdx.z;
  const longlong2 *p = reinterpret_cast<const longlong2 *>(part) + (size_t)tile * nchunks * kMA * kNB + e;
  long long hi = 0, lo = 0;
  for (int c = 0; c < nchunks; ++c) {
    const longlong2 v = p[(size_t)c * kMA * kNB];
    hi += v.x;
    lo += v.y;
  }
  const double val = fix_to_double(hi, lo, FX[a] + FY[b] - 2105);
  double *g = reinterpret_cast<double *>(G + (size_t)a * my + b);
  g[row >> 6] = val;
}

size_t gram_tc_smem_bytes() { return (size_t)2 * kBuf + 64; }

// The dynamic shared-memory limit of kernel `which` raised once per device
// (the attribute is per device).
static void set_smem_attr(const void *func, size_t bytes, int which) {
  static std::atomic<bool> done[2][64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || done[which][dev].load()) return;
  cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  done[which][dev].store(true);
}

int gram_tc_chunks(int n, int mx, int my) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = ceil_div(mx, 64) * ceil_div(my, 64);
  int c = sms / tiles;
  if (c < 1) c = 1;
  const int byrows = ceil_div(n, 4 * kRows);
  return c < byrows ? c : (byrows < 1 ? 1 : byrows);
}

size_t gram_tc_part_bytes(int nchunks, int mx, int my) {
  return (size_t)nchunks * ceil_div(mx, 64) * ceil_div(my, 64) * kMA * kNB * 2 * sizeof(long long);
}

// Largest partial buffer gram_tc needs for any mx, my <= kMaxM0 at this n.
size_t gram_tc_part_max(int n) {
  size_t b = 0;
  for (int m : {64, kMaxM0})
    for (int k : {64, kMaxM0}) b = std::max(b, gram_tc_part_bytes(gram_tc_chunks(n, m, k), m, k));
  return b;
}

// G = X^H Y on the tensor cores.  FXY: 2 * kMaxM0 ints of scratch; part: at
// least gram_tc_part_bytes(nchunks, mx, my) bytes.
void gram_tc(const cxd *X, int ldx, int mx, const cxd *Y, int ldy, int my, int n, cxd *G, long long *part,
             int nchunks, int *FXY, int *err, cudaStream_t s) {
  set_smem_attr(reinterpret_cast<const void *>(k_gram_tc), gram_tc_smem_bytes(), 0);
  int *FX = FXY, *FY = FXY + kMaxM0;
  cudaMemsetAsync(FXY, 0, 2 * kMaxM0 * sizeof(int), s);
  const int erows = 1024;
  k_col_expo<<<dim3(ceil_div(n, erows), 2), 256, 0, s>>>(X, ldx, mx, Y, ldy, my, n, erows, FX, FY);
  note_launch();
  int rpc = ceil_div(ceil_div(n, nchunks), kRows) * kRows;
  const int nc = ceil_div(n, rpc);
  const dim3 grid(nc, ceil_div(mx, 64), ceil_div(my, 64));
  k_gram_tc<<<grid, kThreads, gram_tc_smem_bytes(), s>>>(X, ldx, mx, Y, ldy, my, n, rpc, FX, FY, part, err);
  note_launch();
  k_gram_tc_reduce<<<dim3(kMA * kNB / 256, grid.y, grid.z), 256, 0, s>>>(part, nc, mx, my, FX, FY, G);
  note_launch();
}

// ---------------------------------------------------------------------------
// Z = X S  (n x mx times mx x mz; U = Q V Gamma^{-1/2} of eq. uu, Y = U W of
// step 4.d) with the same exact digit products.  GEMM rows are rows of X,
// with the per-row exponent field F_r of X; GEMM columns (N = 64) are 32
// columns of S in two forms, row c of B' = (Re S[.][c], -Im S[.][c]) for Re Z
// and row 32 + c = (Im S[.][c], Re S[.][c]) for Im Z, with the per-column
// exponent field of S; K = 2 mx interleaved (Re, Im) as X is stored.  A CTA
// takes 128 rows x 32 columns of Z; the exponents are found in the CTA, the
// levels are folded into int64 every 4 stages as above, and the result is
// rounded once to FP64 and staged through shared memory for coalesced stores.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) k_block_tc(const cxd *__restrict__ X, int ldx, int mx,
                                                          const cxd *__restrict__ S, int lds, int mz, int n,
                                                          cxd *__restrict__ Z, int ldz, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * kBuf);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 2 * kBuf + 16);
  int *FR = reinterpret_cast<int *>(smem + 2 * kBuf + 64);  // 128 row exponents
  int *FS = FR + kMA;                                        // 32 column exponents
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = blockIdx.x * kMA, c0 = blockIdx.y * 32;
  const int nst = ceil_div(mx, kRows);

  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
  }
  if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
  // exponent fields: warp w scans rows 8w .. 8w+7; threads 0..31 the columns
  for (int rr = 0; rr < 8; ++rr) {
    const int row = r0 + warp * 8 + rr;
    int em = 0;
    if (row < n)
      for (int a = lane; a < mx; a += 32) {
        const cxd v = X[(size_t)row * ldx + a];
        em = max(em, max(expo_field(v.re), expo_field(v.im)));
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
    if (lane == 0) FR[warp * 8 + rr] = em;
  }
  if (tid < 32) {
    int em = 0;
    if (c0 + tid < mz)
      for (int a = 0; a < mx; ++a) {
        const cxd v = S[(size_t)a * lds + c0 + tid];
        em = max(em, max(expo_field(v.re), expo_field(v.im)));
      }
    FS[tid] = em;
  }
  tc::fence_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;

  auto convert = [&](int st, int buf) {
    unsigned char *Ab = smem + buf * kBuf;
    unsigned char *Bb = Ab + kS * kAPlane;
    const int a0 = st * kRows;
    cxd v[4];
    // A': lanes cover 8 consecutive rows x 4 consecutive k-pairs
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = tid + j * kThreads, w = e >> 5, ln = e & 31;
      const int row = (w & 15) * 8 + (ln & 7), al = (w >> 4) * 4 + (ln >> 3);
      const bool ok = r0 + row < n && a0 + al < mx;
      v[j] = ok ? X[(size_t)(r0 + row) * ldx + a0 + al] : mk(0.0, 0.0);
    }
    const int bal = tid >> 5, bcl = tid & 31;
    const bool bok = a0 + bal < mx && c0 + bcl < mz;
    const cxd sv = bok ? S[(size_t)(a0 + bal) * lds + c0 + bcl] : mk(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = tid + j * kThreads, w = e >> 5, ln = e & 31;
      const int row = (w & 15) * 8 + (ln & 7), al = (w >> 4) * 4 + (ln >> 3);
      int dr[kS], di[kS];
      split_digits(v[j].re, FR[row], dr);
      split_digits(v[j].im, FR[row], di);
      const int o = canon(row, 2 * al);
#pragma unroll
      for (int s = 0; s < kS; ++s) *reinterpret_cast<uint32_t *>(Ab + s * kAPlane + o) = bf16_pair(dr[s], di[s]);
    }
    {
      int dr[kS], di[kS];
      split_digits(sv.re, FS[bcl], dr);
      split_digits(sv.im, FS[bcl], di);
      const int o1 = canon(bcl, 2 * bal), o2 = canon(32 + bcl, 2 * bal);
#pragma unroll
      for (int s = 0; s < kS; ++s) {
        *reinterpret_cast<uint32_t *>(Bb + s * kBPlane + o1) = bf16_pair(dr[s], -di[s]);
        *reinterpret_cast<uint32_t *>(Bb + s * kBPlane + o2) = bf16_pair(di[s], dr[s]);
      }
    }
  };

  long long hi[16], lo[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
  const int q = warp & 3, cg = warp >> 2;

  convert(0, 0);
  tc::fence_smem();
  __syncthreads();
  bool ok = true;
  int issued = 0;
  for (int st = 0; st < nst; ++st) {
    const int b = st & 1;
    if (tid == 0) {
      tc::fence_after();
      const uint32_t abase = tc::smem_u32(smem + b * kBuf), bbase = abase + kS * kAPlane;
      const bool first = (st % kFlush) == 0;
#pragma unroll
      for (int g = 0; g < kS; ++g)
#pragma unroll
        for (int s = 0; s <= g; ++s)
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            tc::mma(tmem + 64 * g, tc::smem_desc(abase + s * kAPlane + kk * 2 * kCoreK, kCoreK, kSBO),
                    tc::smem_desc(bbase + (g - s) * kBPlane + kk * 2 * kCoreK, kCoreK, kSBO), kIdescG,
                    (first && s == 0 && kk == 0) ? 0u : 1u);
      tc::commit(&bar[b]);
    }
    issued = st + 1;
    if (st + 1 < nst) {
      const bool w1 = st >= 1 ? tc::mbar_wait(&bar[b ^ 1], ((st - 1) >> 1) & 1) : true;
      if (__syncthreads_or(!w1)) {
        ok = false;
        break;
      }
      convert(st + 1, b ^ 1);
      tc::fence_smem();
    }
    if (st % kFlush == kFlush - 1 || st == nst - 1) {
      const bool w2 = tc::mbar_wait(&bar[b], (st >> 1) & 1);
      if (__syncthreads_or(!w2)) {
        ok = false;
        break;
      }
      tc::fence_after();
#pragma unroll
      for (int g = 0; g < kS; ++g) {
        float v[16];
        tc::ld16(tmem + ((uint32_t)(q * 32) << 16) + 64 * g + 16 * cg, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const long long iv = f2i_exact(v[c]);
          if (g <= 3)
            hi[c] += iv << (7 * (3 - g));
          else
            lo[c] += iv << (7 * (7 - g));
        }
      }
      tc::fence_before();
    }
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) {
      atomicOr(err, DEVERR_TIMEOUT);
      if (issued >= 1) tc::mbar_wait(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
    }
  } else {
    // all products are done (the last stage flushed): stage Z through buffer 0
    double *Zs = reinterpret_cast<double *>(smem);  // [128][32] complex
    const int row = q * 32 + lane;
    const int part = cg >> 1, cl0 = (cg & 1) * 16;  // part 0: Re, 1: Im
#pragma unroll
    for (int c = 0; c < 16; ++c)
      Zs[((size_t)row * 32 + cl0 + c) * 2 + part] = fix_to_double(hi[c], lo[c], FR[row] + FS[cl0 + c] - 2105);
    __syncthreads();
    for (int e = tid; e < kMA * 32; e += kThreads) {
      const int rr = e >> 5, cc = e & 31;
      if (r0 + rr < n && c0 + cc < mz)
        Z[(size_t)(r0 + rr) * ldz + c0 + cc] = mk(Zs[(size_t)e * 2], Zs[(size_t)e * 2 + 1]);
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_free(tmem, kTmemCols);
}

size_t block_tc_smem_bytes() { return (size_t)2 * kBuf + 64 + (kMA + 32) * sizeof(int); }

void block_tc(const cxd *X, int ldx, int mx, const cxd *S, int lds, int mz, int n, cxd *Z, int ldz, int *err,
              cudaStream_t s) {
  set_smem_attr(reinterpret_cast<const void *>(k_block_tc), block_tc_smem_bytes(), 1);
  const dim3 grid(ceil_div(n, kMA), ceil_div(mz, 32));
  k_block_tc<<<grid, kThreads, block_tc_smem_bytes(), s>>>(X, ldx, mx, S, lds, mz, n, Z, ldz, err);
  note_launch();
}
