// Network of the learned preconditioner: a stack of 3x3 convolutions on the
// N x N grid of the 2-D operator, 32 channels, BF16 weights and activations,
// FP32 accumulation, zero padding at the grid boundary.
//
//   z_l = conv3x3(a_{l-1}; W_l) + b_l,  a_l = relu(z_l) (l < L),  out = z_L
//
// Activations are channel-last (image, y, x, 32 channels): 64 bytes a pixel.
// Weights W_l[tap][c_in][c_out], tap = 3*dy + dx for the offset (dy-1, dx-1).
//
// k_conv3x3_tc: the convolution as an implicit GEMM on the tensor cores.
// A CTA of 128 threads takes tiles of 128 consecutive pixels; per tile
//   D (128 pixels x 32 out-channels, FP32, in tensor memory)
//     = A (128 x 288: the nine shifted 32-channel neighbours of each pixel)
//     x B (288 x 32: the weights),
// with A and B in shared memory in the canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices; LBO = 128 B between core matrices along K,
// SBO = 36 * 128 B between 8-row groups), issued as 18 tcgen05.mma
// (M = 128, N = 32, K = 16, kind::f16 with BF16 operands) by one thread and
// committed to an mbarrier; every warp then reads its 32 rows of D with
// tcgen05.ld and applies the epilogue (bias, ReLU, or the ReLU mask of the
// backward pass) before storing BF16 (and optionally FP32) results.
// The backward data pass is the same kernel with the weights flipped and
// their channel axes swapped; the weight gradient is a CUDA-core reduction
// over pixels (per-CTA partials, fixed-order sum).
#include <algorithm>
#include <cuda_bf16.h>
#include "kernels.h"
#include "tc.cuh"

namespace {

constexpr int kC = 32;               // channels
constexpr int kK = 9 * kC;           // GEMM depth: 288
constexpr int kTile = 128;           // pixels per tile (GEMM M)
constexpr int kLBO = 128;            // bytes between core matrices along K
constexpr int kSBO = (kK / 8) * 128; // bytes between 8-row groups: 4608
constexpr int kAB = kTile * kK * 2;  // A tile bytes: 73728
constexpr int kBB = kC * kK * 2;     // weight bytes: 18432

using tc::smem_u32;
using tc::smem_desc;
using tc::mbar_init;
using tc::mbar_wait;
constexpr uint32_t kIdesc = tc::idesc_bf16(kTile, kC);

// byte offset of element (row, k) in a canonical K-major no-swizzle operand
__device__ __forceinline__ int canon_off(int row, int k) {
  return (row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2;
}

}  // namespace

// out[p][co] = epilogue(sum_{tap, ci} W[tap][ci][co] in[p + off(tap)][ci])
// epilogue: + bias[co] (if bias), relu (if relu), * (mask[p][co] > 0) (if mask);
// stored as BF16 to out (if out) and FP32 to outf (if outf).
__global__ void __launch_bounds__(128, 2) k_conv3x3_tc(const __nv_bfloat16 *__restrict__ in,
                                                       const __nv_bfloat16 *__restrict__ W,
                                                       const float *__restrict__ bias,
                                                       const __nv_bfloat16 *__restrict__ mask, int relu,
                                                       __nv_bfloat16 *__restrict__ out, float *__restrict__ outf,
                                                       int nimg, int N, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *As = smem;
  unsigned char *Bs = smem + kAB;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kAB + kBB);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + kAB + kBB + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  // weights -> canonical B layout (row = out-channel n, k = tap*32 + ci)
  for (int e = tid; e < kK * (kC / 8); e += blockDim.x) {
    const int k = e / (kC / 8), n8 = (e % (kC / 8)) * 8;  // 8 consecutive out-channels of one k
    const int tap = k / kC, ci = k % kC;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const __nv_bfloat16 v = W[((size_t)tap * kC + ci) * kC + n8 + q];
      *reinterpret_cast<__nv_bfloat16 *>(Bs + canon_off(n8 + q, k)) = v;
    }
  }
  if (tid == 0) mbar_init(bar, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const long long npix = (long long)nimg * N * N;
  const long long ntiles = (npix + kTile - 1) / kTile;
  uint32_t phase = 0;
  bool ok = true;
  for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    // ---- im2col of this thread's pixel into the canonical A layout ----
    const long long p = t * kTile + tid;
    int img = 0, y = 0, x = 0;
    const bool live = p < npix;
    if (live) {
      img = (int)(p / ((long long)N * N));
      const int rem = (int)(p - (long long)img * N * N);
      y = rem / N;
      x = rem - y * N;
    }
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      const bool inb = live && yy >= 0 && yy < N && xx >= 0 && xx < N;
      const uint4 *src = reinterpret_cast<const uint4 *>(in + (((size_t)img * N + (inb ? yy : 0)) * N +
                                                               (inb ? xx : 0)) * kC);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 v = inb ? src[q] : make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4 *>(As + canon_off(tid, tap * kC + q * 8)) = v;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // ---- 18 MMAs, K = 16 each ----
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
      for (int s = 0; s < kK / 16; ++s)
        tc::mma(tmem, smem_desc(a0 + s * 2 * kLBO, kLBO, kSBO), smem_desc(b0 + s * 2 * kLBO, kLBO, kSBO), kIdesc,
                s > 0);
      tc::commit(bar);
    }
    // the CTA agrees on the outcome of the bounded wait, so that every thread
    // takes the same path through the barriers below
    const bool waited = mbar_wait(bar, phase);
    if (__syncthreads_or(!waited)) {
      if (tid == 0) atomicOr(err, DEVERR_TIMEOUT);
      ok = false;
    }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue: warp w holds rows (pixels) 32w .. 32w+31 ----
    float v[32];
    tc::ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
    if (live) {
      if (bias) {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] += bias[k];
      }
      if (relu) {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k], 0.f);
      }
      if (mask) {
        const __nv_bfloat16 *mk_ = mask + (size_t)p * kC;
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = __bfloat162float(mk_[k]) > 0.f ? v[k] : 0.f;
      }
      if (out) {
        uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)p * kC);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          __nv_bfloat162 h[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) h[u] = __floats2bfloat162_rn(v[q * 8 + 2 * u], v[q * 8 + 2 * u + 1]);
          dst[q] = *reinterpret_cast<uint4 *>(h);
        }
      }
      if (outf) {
        float4 *dst = reinterpret_cast<float4 *>(outf + (size_t)p * kC);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// Weights of the adjoint convolution: Wt[tap'][co][ci] = W[tap][ci][co] with
// tap' the mirrored tap (offset negated).
__global__ void k_conv_adjoint_weights(const __nv_bfloat16 *W, __nv_bfloat16 *Wt) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 9 * kC * kC; e += gridDim.x * blockDim.x) {
    const int tap = e / (kC * kC), ci = (e / kC) % kC, co = e % kC;
    Wt[((size_t)(8 - tap) * kC + co) * kC + ci] = W[e];
  }
}

// Weight and bias gradients of one layer: dW[tap][ci][co] = sum_p
// a[p + off(tap)][ci] g[p][co], db[co] = sum_p g[p][co].  Each CTA reduces a
// contiguous chunk of pixels into its own partial (thread = (tap, ci), 32
// accumulators); k_net_reduce sums the partials in CTA order.
constexpr int kGradPix = 64;
__global__ void __launch_bounds__(288) k_conv_wgrad(const __nv_bfloat16 *__restrict__ a,
                                                    const __nv_bfloat16 *__restrict__ g, int nimg, int N,
                                                    long long pix_per_cta, float *__restrict__ part) {
  __shared__ float gs[kGradPix][kC];
  const int tid = threadIdx.x;  // tid = tap * 32 + ci
  const int tap = tid / kC, ci = tid % kC;
  const long long npix = (long long)nimg * N * N;
  const long long p0 = blockIdx.x * pix_per_cta, p1 = min(npix, p0 + pix_per_cta);
  float acc[kC];
#pragma unroll
  for (int k = 0; k < kC; ++k) acc[k] = 0.f;
  float bacc = 0.f;
  for (long long pb = p0; pb < p1; pb += kGradPix) {
    const int cnt = (int)min((long long)kGradPix, p1 - pb);
    __syncthreads();
    for (int e = tid; e < kGradPix * kC; e += blockDim.x) {
      const int r = e / kC, c = e % kC;
      gs[r][c] = r < cnt ? __bfloat162float(g[(size_t)(pb + r) * kC + c]) : 0.f;
    }
    __syncthreads();
    for (int r = 0; r < cnt; ++r) {
      const long long p = pb + r;
      const int img = (int)(p / ((long long)N * N));
      const int rem = (int)(p - (long long)img * N * N);
      const int y = rem / N, x = rem - (rem / N) * N;
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      if (yy < 0 || yy >= N || xx < 0 || xx >= N) continue;
      const float av = __bfloat162float(a[(((size_t)img * N + yy) * N + xx) * kC + ci]);
#pragma unroll
      for (int k = 0; k < kC; ++k) acc[k] = fmaf(av, gs[r][k], acc[k]);
    }
    if (tid < kC)
      for (int r = 0; r < cnt; ++r) bacc += gs[r][tid];
  }
  float *o = part + (size_t)blockIdx.x * (9 * kC * kC + kC);
#pragma unroll
  for (int k = 0; k < kC; ++k) o[(size_t)tid * kC + k] = acc[k];
  if (tid < kC) o[9 * kC * kC + tid] = bacc;
}

__global__ void k_net_reduce(const float *part, int nparts, int count, float *out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += part[(size_t)p * count + e];
    out[e] = (float)s;
  }
}

// Loss of the first cout channels against the FP32 target and its gradient
// g = 2 (out - t) / count as BF16 (other channels zero); loss summed in FP64.
__global__ void k_net_loss_grad(const float *__restrict__ out, const float *__restrict__ target, int cout,
                                long long npix, __nv_bfloat16 *__restrict__ g, double *loss) {
  double local = 0.0;
  const double inv = 1.0 / ((double)npix * cout);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < npix * kC;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / kC;
    const int c = (int)(e - p * kC);
    float gv = 0.f;
    if (c < cout) {
      const float d = out[e] - target[p * cout + c];
      local += (double)d * d;
      gv = (float)(2.0 * d * inv);
    }
    g[e] = __float2bfloat16(gv);
  }
  for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, local * inv);
}

// Adam step on FP32 master parameters; BF16 copy of the weights for the
// convolution kernel.  t: step number (1-based).
__global__ void k_net_adam(float *w, const float *grad, float *m1, float *m2, int count, float lr, float b1,
                           float b2, float epsv, int t, __nv_bfloat16 *wb, int nweights) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    const float gr = grad[e];
    m1[e] = b1 * m1[e] + (1.f - b1) * gr;
    m2[e] = b2 * m2[e] + (1.f - b2) * gr * gr;
    w[e] -= lr * (m1[e] / c1) / (sqrtf(m2[e] / c2) + epsv);
    if (e < nweights) wb[e] = __float2bfloat16(w[e]);
  }
}

__global__ void k_to_bf16(const float *x, __nv_bfloat16 *y, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
    y[e] = __float2bfloat16(x[e]);
}
__global__ void k_bf16_to_f32(const __nv_bfloat16 *x, float *y, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
    y[e] = __bfloat162float(x[e]);
}

// Per-system RMS of a node-major block (system s = j*m + c over its n rows):
// per-CTA partial sums of |v|^2, then a fixed-order reduction.
__global__ void k_sys_norm2(const cxf *v, int ne, int n, int m, int rows_per_cta, float *part) {
  const int S = ne * m;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const int j = s / m, c = s - j * m;
    float acc = 0.f;
    for (int i = r0; i < r1; ++i) acc += abs2(v[((size_t)j * n + i) * m + c]);
    part[(size_t)blockIdx.x * S + s] = acc;
  }
}
__global__ void k_sys_rms(const float *part, int nparts, int S, int n, float *rms) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  double a = 0.0;
  for (int p = 0; p < nparts; ++p) a += part[(size_t)p * S + s];
  const double r = sqrt(a / n);
  rms[s] = r > 0 ? (float)r : 1.f;
}
// Image of system s0 + q (q < cnt), pixel i = y N + x: channels
// [Re v / rms, Im v / rms, kappa Re z_j, kappa Im z_j, features..., 0...].
__global__ void k_net_pack(const cxf *v, int ne, int n, int m, int s0, int cnt, const cxd *z, int conj_z, float kappa,
                           const float *feat, int nfeat, const float *rms, __nv_bfloat16 *act) {
  const long long total = (long long)cnt * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e % cnt), i = (int)(e / cnt);  // systems fastest: coalesced reads of v
    const int s = s0 + q, j = s / m, c = s - j * m;
    const cxf val = v[((size_t)j * n + i) * m + c];
    const float inv = 1.f / rms[s];
    cxd zz = z[j];
    if (conj_z) zz = conj(zz);
    float ch[kC];
#pragma unroll
    for (int k = 0; k < kC; ++k) ch[k] = 0.f;
    ch[0] = val.re * inv;
    ch[1] = val.im * inv;
    ch[2] = kappa * (float)zz.re;
    ch[3] = kappa * (float)zz.im;
    for (int k = 0; k < nfeat && k < kC - 4; ++k) ch[4 + k] = feat[k];
    uint4 *dst = reinterpret_cast<uint4 *>(act + ((size_t)q * n + i) * kC);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      __nv_bfloat162 h[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) h[w] = __floats2bfloat162_rn(ch[u * 8 + 2 * w], ch[u * 8 + 2 * w + 1]);
      dst[u] = *reinterpret_cast<uint4 *>(h);
    }
  }
}
// z (system s0 + q) = rms * (out0 + i out1)
__global__ void k_net_unpack(const float *outf, int ne, int n, int m, int s0, int cnt, const float *rms, cxf *z) {
  const long long total = (long long)cnt * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e % cnt), i = (int)(e / cnt);
    const int s = s0 + q, j = s / m, c = s - j * m;
    const float2 o = *reinterpret_cast<const float2 *>(outf + ((size_t)q * n + i) * kC);
    z[((size_t)j * n + i) * m + c] = mk(rms[s] * o.x, rms[s] * o.y);
  }
}

// Training pairs from exact solves.  Inputs: the image of system s = (j, c)
// is column c of R (shared by the nodes) packed as the preconditioner packs
// its input (Re, Im over the column's RMS, kappa z_j, features), FP32.
// Targets: X_j[:, c] over its own RMS (the direction of the correction).
__global__ void k_pairs_inputs(const cxd *R, int ne, int n, int m, const cxd *z, float kappa, const float *feat,
                               int nfeat, const double *rn2, float *Xin) {
  const long long total = (long long)ne * m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / n), i = (int)(e - (long long)s * n);
    const int j = s / m, c = s - j * m;
    const double rms = sqrt(rn2[c] / n);
    const double inv = rms > 0 ? 1.0 / rms : 1.0;
    const cxd v = R[(size_t)i * m + c];
    float *o = Xin + ((size_t)s * n + i) * kC;
    o[0] = (float)(v.re * inv);
    o[1] = (float)(v.im * inv);
    o[2] = kappa * (float)z[j].re;
    o[3] = kappa * (float)z[j].im;
    for (int k = 4; k < kC; ++k) o[k] = (k - 4 < nfeat) ? feat[k - 4] : 0.f;
  }
}
// targets: the node solution for the normalised column, X_j[:, c] / rms(R[:, c])
__global__ void k_pairs_targets(const cxd *X, int ne, int n, int m, const double *rn2, float *T) {
  const long long total = (long long)ne * m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / n), i = (int)(e - (long long)s * n);
    const int j = s / m, c = s - j * m;
    const double rms = sqrt(rn2[c] / n);
    const double inv = rms > 0 ? 1.0 / rms : 1.0;
    const cxd v = X[((size_t)j * n + i) * m + c];
    T[((size_t)s * n + i) * 2] = (float)(v.re * inv);
    T[((size_t)s * n + i) * 2 + 1] = (float)(v.im * inv);
  }
}
void launch_learned_pairs(const cxd *R, const cxd *X, int ne, int n, int m, const cxd *z, float kappa,
                          const float *feat, int nfeat, const double *rn2, float *Xin, float *T, cudaStream_t s) {
  k_pairs_inputs<<<grid_for((size_t)ne * m * n), 256, 0, s>>>(R, ne, n, m, z, kappa, feat, nfeat, rn2, Xin);
  note_launch();
  k_pairs_targets<<<grid_for((size_t)ne * m * n), 256, 0, s>>>(X, ne, n, m, rn2, T);
  note_launch();
}

// Operator-norm loss of the network output against exact corrections: for
// system s = (j, c), d = out_s - T_s (channels 0, 1 as a complex image),
// y = (z_j I - A) d (the node's shifted operator applied on the grid; conj(z_j)
// and A^H for side 1), loss = sum |y|^2 / count, and its gradient with
// respect to out, g = 2 (z_j I - A)^H y / count, written to channels 0, 1 of
// gout (32 channels, others zero).  With T the exact correction of the input
// residual, y = (z_j I - A) out_s - r_s.
__global__ void k_oploss_apply(CsrView M, int ne, int n, int m, const cxd *z, int conj_z, const float *out,
                               const float *T, float *y, double *loss) {
  const long long total = (long long)ne * m * n;
  double local = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / n), i = (int)(e - (long long)s * n);
    const int j = s / m;
    cxd zj = z[j];
    if (conj_z) zj = conj(zj);
    auto dval = [&](int k) {
      const float *o = out + ((size_t)s * n + k) * 32;
      const float *t = T + ((size_t)s * n + k) * 2;
      return mk((double)o[0] - t[0], (double)o[1] - t[1]);
    };
    cxd acc = zj * dval(i);
    for (int64_t k = M.rowptr[i]; k < M.rowptr[i + 1]; ++k) cfms(acc, csr_val(M, k), dval(M.colind[k]));
    y[((size_t)s * n + i) * 2] = (float)acc.re;
    y[((size_t)s * n + i) * 2 + 1] = (float)acc.im;
    local += abs2(acc);
  }
  for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, local / (double)total);
}
__global__ void k_oploss_grad(CsrView MH, int ne, int n, int m, const cxd *z, int conj_z, const float *y,
                              float *gout) {
  const long long total = (long long)ne * m * n;
  const double sc = 2.0 / (double)total;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / n), i = (int)(e - (long long)s * n);
    const int j = s / m;
    cxd zj = z[j];
    if (!conj_z) zj = conj(zj);  // adjoint of (z I - A) is (conj z I - A^H)
    auto yv = [&](int k) {
      const float *q = y + ((size_t)s * n + k) * 2;
      return mk((double)q[0], (double)q[1]);
    };
    cxd acc = zj * yv(i);
    for (int64_t k = MH.rowptr[i]; k < MH.rowptr[i + 1]; ++k) cfms(acc, csr_val(MH, k), yv(MH.colind[k]));
    float *g = gout + ((size_t)s * n + i) * 32;
    g[0] = (float)(sc * acc.re);
    g[1] = (float)(sc * acc.im);
    for (int k = 2; k < 32; ++k) g[k] = 0.f;
  }
}
void launch_operator_loss(const CsrView &M, const CsrView &MH, int ne, int n, int m, const cxd *z, int side,
                          const float *out, const float *T, float *ybuf, float *gout, double *loss, cudaStream_t s) {
  k_oploss_apply<<<grid_for((size_t)ne * m * n), 256, 0, s>>>(M, ne, n, m, z, side, out, T, ybuf, loss);
  note_launch();
  k_oploss_grad<<<grid_for((size_t)ne * m * n), 256, 0, s>>>(MH, ne, n, m, z, side, ybuf, gout);
  note_launch();
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
size_t conv_tc_smem_bytes() { return (size_t)kAB + kBB + 64; }

cudaError_t launch_conv3x3_tc(const void *in, const void *W, const float *bias, const void *mask, int relu, void *out,
                              float *outf, int nimg, int N, int *err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)conv_tc_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = ((long long)nimg * N * N + kTile - 1) / kTile;
  long long g = (long long)sms * 2;
  if (g > ntiles) g = ntiles;
  if (g < 1) g = 1;
  k_conv3x3_tc<<<(unsigned)g, kTile, conv_tc_smem_bytes(), s>>>(
      (const __nv_bfloat16 *)in, (const __nv_bfloat16 *)W, bias, (const __nv_bfloat16 *)mask, relu,
      (__nv_bfloat16 *)out, outf, nimg, N, err);
  note_launch();
  return cudaGetLastError();
}

void launch_conv_adjoint_weights(const void *W, void *Wt, cudaStream_t s) {
  k_conv_adjoint_weights<<<ceil_div(9 * kC * kC, 256), 256, 0, s>>>((const __nv_bfloat16 *)W, (__nv_bfloat16 *)Wt);
  note_launch();
}

int conv_wgrad_parts(long long npix) {
  long long p = (npix + 4095) / 4096;
  if (p > 1216) p = 1216;
  return (int)(p < 1 ? 1 : p);
}

void launch_conv_wgrad(const void *a, const void *g, int nimg, int N, float *part, float *dWb, cudaStream_t s) {
  const long long npix = (long long)nimg * N * N;
  const int parts = conv_wgrad_parts(npix);
  const long long per = (npix + parts - 1) / parts;
  k_conv_wgrad<<<parts, 288, 0, s>>>((const __nv_bfloat16 *)a, (const __nv_bfloat16 *)g, nimg, N, per, part);
  note_launch();
  const int count = 9 * kC * kC + kC;
  k_net_reduce<<<ceil_div(count, 256), 256, 0, s>>>(part, parts, count, dWb);
  note_launch();
}

void launch_net_loss_grad(const float *out, const float *target, int cout, long long npix, void *g, double *loss,
                          cudaStream_t s) {
  k_net_loss_grad<<<grid_for((size_t)npix * kC), 256, 0, s>>>(out, target, cout, npix, (__nv_bfloat16 *)g, loss);
  note_launch();
}

void launch_net_adam(float *w, const float *grad, float *m1, float *m2, int count, float lr, int t, void *wb,
                     int nweights, cudaStream_t s) {
  k_net_adam<<<ceil_div(count, 256), 256, 0, s>>>(w, grad, m1, m2, count, lr, 0.9f, 0.999f, 1e-8f, t,
                                                  (__nv_bfloat16 *)wb, nweights);
  note_launch();
}

void launch_to_bf16(const float *x, void *y, long long count, cudaStream_t s) {
  k_to_bf16<<<grid_for((size_t)count), 256, 0, s>>>(x, (__nv_bfloat16 *)y, count);
  note_launch();
}
void launch_bf16_to_f32(const void *x, float *y, long long count, cudaStream_t s) {
  k_bf16_to_f32<<<grid_for((size_t)count), 256, 0, s>>>((const __nv_bfloat16 *)x, y, count);
  note_launch();
}

// ---------------------------------------------------------------------------
// network object (C ABI in feast_nh.h)
// ---------------------------------------------------------------------------
#include <algorithm>
#include <string>
#include <vector>
#include "feast_nh.h"

struct feast_nh_net {
  int L = 0, N = 0, maxi = 0, t = 0;
  cudaStream_t s = nullptr;
  std::vector<void *> allocs;
  float *params = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  __nv_bfloat16 *wb = nullptr, *wt = nullptr;
  std::vector<__nv_bfloat16 *> act;  // act[0]: input, act[l]: output of layer l - 1
  float *outf = nullptr;
  __nv_bfloat16 *g0 = nullptr, *g1 = nullptr;
  float *wpart = nullptr;
  double *dloss = nullptr;
  int *derr = nullptr;
  std::string err;
};

namespace {
constexpr int kLayerP = 9 * kC * kC + kC;  // parameters per layer: W then b
constexpr int kLayerW = 9 * kC * kC;

template <typename P>
P *nalloc(feast_nh_net *n, size_t bytes, bool &ok) {
  void *p = nullptr;
  if (!ok) return nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
    ok = false;
    return nullptr;
  }
  n->allocs.push_back(p);
  return reinterpret_cast<P *>(p);
}

void net_free(feast_nh_net *n) {
  if (!n) return;
  if (n->s) cudaStreamSynchronize(n->s);
  for (void *p : n->allocs) cudaFree(p);
  delete n;
}

feast_nh_status net_forward(feast_nh_net *n, int nimg) {
  for (int l = 0; l < n->L; ++l) {
    const bool last = l == n->L - 1;
    const cudaError_t e =
        launch_conv3x3_tc(n->act[l], n->wb + (size_t)l * kLayerW, n->params + (size_t)l * kLayerP + kLayerW, nullptr,
                          last ? 0 : 1, last ? nullptr : n->act[l + 1], last ? n->outf : nullptr, nimg, n->N, n->derr,
                          n->s);
    if (e != cudaSuccess) {
      n->err = std::string("network forward: ") + cudaGetErrorString(e);
      return FEAST_NH_ECUDA;
    }
  }
  return FEAST_NH_OK;
}

feast_nh_status net_check(feast_nh_net *n) {
  int herr = 0;
  if (cudaMemcpyAsync(&herr, n->derr, sizeof(int), cudaMemcpyDeviceToHost, n->s) != cudaSuccess ||
      cudaStreamSynchronize(n->s) != cudaSuccess) {
    n->err = "network: CUDA error";
    return FEAST_NH_ECUDA;
  }
  if (herr & DEVERR_TIMEOUT) {
    n->err = "network: a bounded wait for the tensor-core product gave up";
    return FEAST_NH_ETIMEOUT;
  }
  return FEAST_NH_OK;
}
}  // namespace

// forward of the network on nimg bf16 channel-last images already in act[0]
// (used by the preconditioned Krylov solver)
feast_nh_status net_apply_internal(feast_nh_net *n, int nimg, const float **out) {
  if (nimg > n->maxi) return FEAST_NH_EINVAL;
  const feast_nh_status st = net_forward(n, nimg);
  *out = n->outf;
  return st;
}
void *net_input_buffer(feast_nh_net *n) { return n->act[0]; }

// z = network(v) for every system of a node-major block (images of the
// N x N grid, n = N^2), in chunks of at most max_images systems.
int net_precondition(feast_nh_net *net, const cxf *v, cxf *z, int ne, int n, int m, const cxd *zn,
                                 int conj_z, float kappa, const float *feat, int nfeat, float *part, float *rms,
                                 cudaStream_t s) {
  if ((long long)net->N * net->N != n) return FEAST_NH_EINVAL;
  const int S = ne * m;
  const int parts = std::min(1216, n);
  const int rpc = ceil_div(n, parts), np = ceil_div(n, rpc);
  k_sys_norm2<<<np, 256, 0, s>>>(v, ne, n, m, rpc, part);
  note_launch();
  k_sys_rms<<<ceil_div(S, 256), 256, 0, s>>>(part, np, S, n, rms);
  note_launch();
  for (int s0 = 0; s0 < S; s0 += net->maxi) {
    const int cnt = std::min(net->maxi, S - s0);
    k_net_pack<<<grid_for((size_t)cnt * n), 256, 0, s>>>(v, ne, n, m, s0, cnt, zn, conj_z, kappa, feat, nfeat, rms,
                                                         net->act[0]);
    note_launch();
    cudaStream_t keep = net->s;
    net->s = s;
    const feast_nh_status st = net_forward(net, cnt);
    net->s = keep;
    if (st != FEAST_NH_OK) return st;
    k_net_unpack<<<grid_for((size_t)cnt * n), 256, 0, s>>>(net->outf, ne, n, m, s0, cnt, rms, z);
    note_launch();
  }
  return FEAST_NH_OK;
}
size_t net_precondition_scratch_floats(int n, int ne, int m) { return (size_t)std::min(1216, n) * ne * m + ne * m; }
int *net_error_word(feast_nh_net *n) { return n->derr; }
int net_grid(const feast_nh_net *n) { return n->N; }
int net_max_images(const feast_nh_net *n) { return n->maxi; }

extern "C" {

feast_nh_status feast_nh_net_create(feast_nh_net **out, int32_t layers, int32_t N, int32_t max_images,
                                    void *stream) {
  if (!out) return FEAST_NH_EINVAL;
  *out = nullptr;
  if (layers < 1 || layers > 16 || N < 2 || max_images < 1) return FEAST_NH_EINVAL;
  feast_nh_net *n = new feast_nh_net();
  n->L = layers;
  n->N = N;
  n->maxi = max_images;
  n->s = reinterpret_cast<cudaStream_t>(stream);
  bool ok = true;
  const size_t np = (size_t)layers * kLayerP;
  const size_t pix = (size_t)max_images * N * N;
  n->params = nalloc<float>(n, np * sizeof(float), ok);
  n->grad = nalloc<float>(n, np * sizeof(float), ok);
  n->m1 = nalloc<float>(n, np * sizeof(float), ok);
  n->m2 = nalloc<float>(n, np * sizeof(float), ok);
  n->wb = nalloc<__nv_bfloat16>(n, (size_t)layers * kLayerW * 2, ok);
  n->wt = nalloc<__nv_bfloat16>(n, (size_t)kLayerW * 2, ok);
  n->act.assign(layers, nullptr);
  for (int l = 0; l < layers; ++l) n->act[l] = nalloc<__nv_bfloat16>(n, pix * kC * 2, ok);
  n->outf = nalloc<float>(n, pix * kC * sizeof(float), ok);
  n->g0 = nalloc<__nv_bfloat16>(n, pix * kC * 2, ok);
  n->g1 = nalloc<__nv_bfloat16>(n, pix * kC * 2, ok);
  n->wpart = nalloc<float>(n, (size_t)conv_wgrad_parts((long long)pix) * kLayerP * sizeof(float), ok);
  n->dloss = nalloc<double>(n, sizeof(double), ok);
  n->derr = nalloc<int>(n, sizeof(int), ok);
  if (!ok) {
    net_free(n);
    return FEAST_NH_ENOMEM;
  }
  if (cudaMemsetAsync(n->params, 0, np * sizeof(float), n->s) != cudaSuccess ||
      cudaMemsetAsync(n->m1, 0, np * sizeof(float), n->s) != cudaSuccess ||
      cudaMemsetAsync(n->m2, 0, np * sizeof(float), n->s) != cudaSuccess ||
      cudaMemsetAsync(n->wb, 0, (size_t)layers * kLayerW * 2, n->s) != cudaSuccess ||
      cudaMemsetAsync(n->derr, 0, sizeof(int), n->s) != cudaSuccess ||
      cudaStreamSynchronize(n->s) != cudaSuccess) {
    net_free(n);
    return FEAST_NH_ECUDA;
  }
  *out = n;
  return FEAST_NH_OK;
}

void feast_nh_net_destroy(feast_nh_net *n) { net_free(n); }

const char *feast_nh_net_last_error(const feast_nh_net *n) { return n ? n->err.c_str() : ""; }

feast_nh_status feast_nh_net_set_params(feast_nh_net *n, const float *params) {
  if (!n || !params) return FEAST_NH_EINVAL;
  const size_t np = (size_t)n->L * kLayerP;
  if (cudaMemcpyAsync(n->params, params, np * sizeof(float), cudaMemcpyHostToDevice, n->s) != cudaSuccess)
    return FEAST_NH_ECUDA;
  for (int l = 0; l < n->L; ++l)
    launch_to_bf16(n->params + (size_t)l * kLayerP, n->wb + (size_t)l * kLayerW, kLayerW, n->s);
  cudaMemsetAsync(n->m1, 0, np * sizeof(float), n->s);
  cudaMemsetAsync(n->m2, 0, np * sizeof(float), n->s);
  n->t = 0;
  return cudaStreamSynchronize(n->s) == cudaSuccess ? FEAST_NH_OK : FEAST_NH_ECUDA;
}

feast_nh_status feast_nh_net_get_params(feast_nh_net *n, float *params) {
  if (!n || !params) return FEAST_NH_EINVAL;
  if (cudaMemcpyAsync(params, n->params, (size_t)n->L * kLayerP * sizeof(float), cudaMemcpyDeviceToHost, n->s) !=
          cudaSuccess ||
      cudaStreamSynchronize(n->s) != cudaSuccess)
    return FEAST_NH_ECUDA;
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_net_forward(feast_nh_net *n, const float *x, float *out, int32_t nimg) {
  if (!n || !x || !out || nimg < 1 || nimg > n->maxi) return FEAST_NH_EINVAL;
  const long long cnt = (long long)nimg * n->N * n->N * kC;
  cudaMemsetAsync(n->derr, 0, sizeof(int), n->s);
  launch_to_bf16(x, n->act[0], cnt, n->s);
  feast_nh_status st = net_forward(n, nimg);
  if (st != FEAST_NH_OK) return st;
  if (cudaMemcpyAsync(out, n->outf, cnt * sizeof(float), cudaMemcpyDeviceToDevice, n->s) != cudaSuccess)
    return FEAST_NH_ECUDA;
  return net_check(n);
}

// Backward pass from dL/d out (FP32, 32 channels) through the activations of
// the last forward call, then an optional Adam step.
static feast_nh_status net_backward(feast_nh_net *n, __nv_bfloat16 *g, int nimg, float lr, float *grad_out) {
  cudaStream_t s = n->s;
  __nv_bfloat16 *gn = (g == n->g0) ? n->g1 : n->g0;
  for (int l = n->L - 1; l >= 0; --l) {
    launch_conv_wgrad(n->act[l], g, nimg, n->N, n->wpart, n->grad + (size_t)l * kLayerP, s);
    if (l > 0) {
      launch_conv_adjoint_weights(n->wb + (size_t)l * kLayerW, n->wt, s);
      const cudaError_t e = launch_conv3x3_tc(g, n->wt, nullptr, n->act[l], 0, gn, nullptr, nimg, n->N, n->derr, s);
      if (e != cudaSuccess) {
        n->err = std::string("network backward: ") + cudaGetErrorString(e);
        return FEAST_NH_ECUDA;
      }
      std::swap(g, gn);
    }
  }
  if (grad_out &&
      cudaMemcpyAsync(grad_out, n->grad, (size_t)n->L * kLayerP * sizeof(float), cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return FEAST_NH_ECUDA;
  if (lr > 0) {
    ++n->t;
    for (int l = 0; l < n->L; ++l)
      launch_net_adam(n->params + (size_t)l * kLayerP, n->grad + (size_t)l * kLayerP, n->m1 + (size_t)l * kLayerP,
                      n->m2 + (size_t)l * kLayerP, kLayerP, lr, n->t, n->wb + (size_t)l * kLayerW, kLayerW, s);
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_net_backward(feast_nh_net *n, const float *gout, int32_t nimg, float lr, float *grad) {
  if (!n || !gout || nimg < 1 || nimg > n->maxi || lr < 0) return FEAST_NH_EINVAL;
  const long long npix = (long long)nimg * n->N * n->N;
  cudaMemsetAsync(n->derr, 0, sizeof(int), n->s);
  launch_to_bf16(gout, n->g0, npix * kC, n->s);
  const feast_nh_status st = net_backward(n, n->g0, nimg, lr, grad);
  if (st != FEAST_NH_OK) return st;
  return net_check(n);
}

feast_nh_status feast_nh_net_train_step(feast_nh_net *n, const float *x, const float *target, int32_t cout,
                                        int32_t nimg, float lr, double *loss, float *grad_out) {
  if (!n || !x || !target || cout < 1 || cout > kC || nimg < 1 || nimg > n->maxi || lr < 0) return FEAST_NH_EINVAL;
  cudaStream_t s = n->s;
  const long long npix = (long long)nimg * n->N * n->N;
  cudaMemsetAsync(n->derr, 0, sizeof(int), s);
  cudaMemsetAsync(n->dloss, 0, sizeof(double), s);
  launch_to_bf16(x, n->act[0], npix * kC, s);
  feast_nh_status st = net_forward(n, nimg);
  if (st != FEAST_NH_OK) return st;
  launch_net_loss_grad(n->outf, target, cout, npix, n->g0, n->dloss, s);
  st = net_backward(n, n->g0, nimg, lr, grad_out);
  if (st != FEAST_NH_OK) return st;
  if (loss && cudaMemcpyAsync(loss, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return FEAST_NH_ECUDA;
  return net_check(n);
}

}  // extern "C"
