// E4M3 operands of the low-rank Casida matvec.
//
// Two ways of using E4M3 L: both operands E4M3 (kind::f8f6f4), or L alone in
// E4M3, widened to FP16 in shared memory against FP16 operands x16 and y16
// (kind::f16); the scales are the same, with FP16 in place of E4M3 for the
// per-step operands.
//
// L is stored as L8 = e4m3(L / s_mu) with one power-of-two scale per column
// mu (s_mu = 2^ceil(log2(max_vc |L[vc][mu]| / 448)), so the largest entry
// maps into (224, 448] and dequantisation is exact); both row-major copies
// L8 [N][A] (K = N_aux contiguous, gemm2) and L8t [A][N] (K = N_vc, gemm1,
// K-block-major like x8).
// Per Lanczos step:
//   x8 = e4m3(Delta^1/2 q / s_b)       s_b per vector (k_quant_x8)
//   Y^T[mu][b] = s_b s_mu sum_vc L8t[mu][vc] x8[b][vc]     (tensor cores)
//   y'_mu = s_mu y_mu,  y8 = e4m3(y' / t_b)                  (k_reduce_y_fp8)
//   U[vc][b] = t_b sum_mu L8[vc][mu] y8[b][mu]               (tensor cores)
// so U = (s L8)(t y8 / s) ~ L y.  The FP64 recurrence is unchanged.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lgw_internal.cuh"

namespace lgw {

__device__ __forceinline__ float pow2_scale(float amax, float top = 448.0f) {
  // smallest power of two s with amax / s <= top
  if (!(amax > 0.0f)) return 1.0f;
  int e;
  const float m = frexpf(amax / top, &e);   // amax/top = m 2^e, m in [0.5, 1)
  if (m == 0.5f) e -= 1;
  return ldexpf(1.0f, e);
}

// FP16 operands of the widening path are scaled per vector so that the
// largest magnitude lands in (2^14, 2^15]: far from FP16 overflow (65504)
// and with 2^-24 / 2^-15 = 2^-9 of headroom before values turn subnormal.
constexpr float F16_TOP = 32768.0f;

__device__ __forceinline__ uint8_t to_e4m3(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ float from_e4m3(uint8_t v) {
  const __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)v, __NV_E4M3);
  return __half2float(__half(hr));
}

// column maxima of |L| over L [nr][nc] (row stride ld); non-negative floats
// order like their bit patterns
__global__ void k_col_absmax(const double *__restrict__ src, int ld, int nr, int nc,
                             unsigned *__restrict__ colmax) {
  __shared__ float red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int mu = blockIdx.x * 32 + tx;
  const int r0 = blockIdx.y * 1024;
  float m = 0.0f;
  if (mu < nc)
    for (int r = r0 + ty; r < min(nr, r0 + 1024); r += 8)
      m = fmaxf(m, (float)fabs(src[(size_t)r * ld + mu]));
  red[ty][tx] = m;
  __syncthreads();
  if (ty == 0 && mu < nc) {
    for (int i = 1; i < 8; ++i) m = fmaxf(m, red[i][tx]);
    atomicMax(colmax + mu, __float_as_uint(m));
  }
}

__global__ void k_col_scales(const unsigned *__restrict__ colmax, int A, float *__restrict__ sL) {
  const int mu = blockIdx.x * blockDim.x + threadIdx.x;
  if (mu < A) sL[mu] = pow2_scale(__uint_as_float(colmax[mu]));
}

// L8 = e4m3(L / s_mu) [N][A] from L [nr][nc] (row stride ld, zero padded)
// and its transpose L8t [A][N], K-block-major (32 x 32 tiles)
__global__ void k_quantize_L8(const double *__restrict__ src, int ld, int nr, int nc, int N, int A,
                              const float *__restrict__ sL, uint8_t *__restrict__ L8,
                              uint8_t *__restrict__ L8t) {
  __shared__ uint8_t tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int rr = ty; rr < 32; rr += 8) {
    const int r = r0 + rr, c = c0 + tx;
    uint8_t v = 0;
    if (r < N && c < A) {
      const double x = (r < nr && c < nc) ? src[(size_t)r * ld + c] : 0.0;
      v = to_e4m3((float)(x / (double)sL[c]));
      L8[(size_t)r * A + c] = v;
    }
    tile[rr][tx] = v;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += 8) {
    const int c = c0 + cc, r = r0 + tx;
    if (r < N && c < A) L8t[kblk_e4m3(c, r, A)] = tile[tx][cc];
  }
}

// x8[b] = e4m3(xh[b] / s_b), s_b from max |xh[b]|; one block per vector.
// Both operands are K-block-major over Bs rows.
__global__ void __launch_bounds__(256) k_quant_x8(const __nv_bfloat16 *__restrict__ xh, int Bs,
                                                  int N, uint8_t *__restrict__ x8,
                                                  float *__restrict__ sx,
                                                  const double *__restrict__ vscale) {
  __shared__ float red[8];
  __shared__ float sc;
  const int b = blockIdx.x;
  // eight consecutive elements per thread: one 16-byte load of xh, one
  // 8-byte store of x8 (N is a multiple of 128, so a group never straddles
  // a K block)
  float m = 0.0f;
  for (int g = threadIdx.x; g < N / 8; g += 256) {
    const uint4 v = *reinterpret_cast<const uint4 *>(xh + kblk_bf16(b, 8 * g, Bs));
    const __nv_bfloat162 *p2 = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 f = __bfloat1622float2(p2[t]);
      m = fmaxf(m, fmaxf(fabsf(f.x), fabsf(f.y)));
    }
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t = fmaxf(t, red[w]);
    sc = pow2_scale(t);
    // the contraction result is scaled by sx; an unnormalised operand also
    // carries its normalisation factor there (sx then need not be a power
    // of two: it only multiplies the FP32 reduction)
    sx[b] = vscale != nullptr ? sc * (float)vscale[b] : sc;
  }
  __syncthreads();
  const float inv = 1.0f / sc;   // a power of two: exact
  for (int g = threadIdx.x; g < N / 8; g += 256) {
    const uint4 v = *reinterpret_cast<const uint4 *>(xh + kblk_bf16(b, 8 * g, Bs));
    const __nv_bfloat162 *p2 = reinterpret_cast<const __nv_bfloat162 *>(&v);
    uint32_t wq[2] = {0u, 0u};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 f = __bfloat1622float2(p2[t]);
      const uint32_t lo = to_e4m3(f.x * inv), hi = to_e4m3(f.y * inv);
      wq[t >> 1] |= (lo | (hi << 8)) << (16 * (t & 1));
    }
    *reinterpret_cast<uint2 *>(x8 + kblk_e4m3(b, 8 * g, Bs)) = make_uint2(wq[0], wq[1]);
  }
}

// From the split-K partials of gemm1: y_mu = s_b s_mu sum_p Ypart, then
// y8 = e4m3(s_mu y_mu / t_b) with t_b from the vector's max; yy[b] (slot 0
// of n_yb) = sum_mu y_mu yhat_mu with yhat = t_b y8 / s_mu, the y that gemm2
// effectively multiplies (for the alpha estimate).  One block per vector;
// dynamic shared memory A floats.
__global__ void __launch_bounds__(256) k_reduce_y_fp8(const float *__restrict__ Ypart, int splits,
                                                      int Bs, int A, const float *__restrict__ sx,
                                                      const float *__restrict__ sL,
                                                      uint8_t *__restrict__ y8,
                                                      float *__restrict__ ty,
                                                      float *__restrict__ yy, int n_yb) {
  extern __shared__ float yp[];   // [A]: s_mu y_mu
  __shared__ float red[8];
  __shared__ float sc;
  const int b = blockIdx.x;
  const size_t n = (size_t)Bs * A;
  float m = 0.0f;
  for (int mu = threadIdx.x; mu < A; mu += 256) {
    float s = 0.0f;
    for (int p = 0; p < splits; ++p) s += Ypart[(size_t)p * n + (size_t)b * A + mu];
    const float v = sL[mu] * (sx[b] * sL[mu] * s);
    yp[mu] = v;
    m = fmaxf(m, fabsf(v));
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t = fmaxf(t, red[w]);
    sc = pow2_scale(t);
    ty[b] = sc;
  }
  __syncthreads();
  const float t = sc, inv = 1.0f / sc;
  float acc = 0.0f;
  for (int mu = threadIdx.x; mu < A; mu += 256) {
    const uint8_t q = to_e4m3(yp[mu] * inv);
    y8[(size_t)b * A + mu] = q;
    const float yv = yp[mu] / sL[mu];            // y_mu (exact: s_mu is a power of two)
    acc = fmaf(yv, t * from_e4m3(q) / sL[mu], acc);
  }
  if (yy != nullptr) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float tot = 0.0f;
      for (int w = 0; w < 8; ++w) tot += red[w];
      yy[(size_t)b * n_yb] = tot;
      for (int i = 1; i < n_yb; ++i) yy[(size_t)b * n_yb + i] = 0.0f;
    }
  }
}

// x16[b] = fp16(xh[b] / s_b) with s_b from max |xh[b]| (largest value into
// (2^14, 2^15]; a BF16 value scaled by a power of two is exact in FP16 down
// to 2^-14); one block per vector, K-block-major like xh.
__global__ void __launch_bounds__(256) k_quant_x16(const __nv_bfloat16 *__restrict__ xh, int Bs,
                                                   int N, uint16_t *__restrict__ x16,
                                                   float *__restrict__ sx,
                                                   const double *__restrict__ vscale) {
  __shared__ float red[8];
  __shared__ float sc;
  const int b = blockIdx.x;
  float m = 0.0f;
  for (int g = threadIdx.x; g < N / 8; g += 256) {
    const uint4 v = *reinterpret_cast<const uint4 *>(xh + kblk_bf16(b, 8 * g, Bs));
    const __nv_bfloat162 *p2 = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 f = __bfloat1622float2(p2[t]);
      m = fmaxf(m, fmaxf(fabsf(f.x), fabsf(f.y)));
    }
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t = fmaxf(t, red[w]);
    sc = pow2_scale(t, F16_TOP);
    sx[b] = vscale != nullptr ? sc * (float)vscale[b] : sc;
  }
  __syncthreads();
  const float inv = 1.0f / sc;   // a power of two: exact
  for (int g = threadIdx.x; g < N / 8; g += 256) {
    const size_t o = kblk_bf16(b, 8 * g, Bs);
    const uint4 v = *reinterpret_cast<const uint4 *>(xh + o);
    const __nv_bfloat162 *p2 = reinterpret_cast<const __nv_bfloat162 *>(&v);
    uint32_t w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 f = __bfloat1622float2(p2[t]);
      const __half2 h = __floats2half2_rn(f.x * inv, f.y * inv);
      w[t] = *reinterpret_cast<const uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(x16 + o) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// From the split-K partials of gemm1 on (E4M3 L^T) x16: y_mu = s_b s_mu
// sum_p Ypart, then y16 = fp16(s_mu y_mu / t_b) with t_b from the vector's
// max; yy[b] = sum_mu y_mu yhat_mu with yhat = t_b y16 / s_mu, the y that
// gemm2 effectively multiplies.  One block per vector; dynamic shared
// memory A floats.
__global__ void __launch_bounds__(256) k_reduce_y_f16(const float *__restrict__ Ypart, int splits,
                                                      int Bs, int A, const float *__restrict__ sx,
                                                      const float *__restrict__ sL,
                                                      uint16_t *__restrict__ y16,
                                                      float *__restrict__ ty,
                                                      float *__restrict__ yy, int n_yb) {
  extern __shared__ float yp[];   // [A]: s_mu y_mu
  __shared__ float red[8];
  __shared__ float sc;
  const int b = blockIdx.x;
  const size_t n = (size_t)Bs * A;
  float m = 0.0f;
  for (int mu = threadIdx.x; mu < A; mu += 256) {
    float s = 0.0f;
    for (int p = 0; p < splits; ++p) s += Ypart[(size_t)p * n + (size_t)b * A + mu];
    const float v = sL[mu] * (sx[b] * sL[mu] * s);
    yp[mu] = v;
    m = fmaxf(m, fabsf(v));
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t = fmaxf(t, red[w]);
    sc = pow2_scale(t, F16_TOP);
    ty[b] = sc;
  }
  __syncthreads();
  const float t = sc, inv = 1.0f / sc;
  float acc = 0.0f;
  for (int mu = threadIdx.x; mu < A; mu += 256) {
    const __half q = __float2half_rn(yp[mu] * inv);
    y16[(size_t)b * A + mu] = __half_as_ushort(q);
    const float yv = yp[mu] / sL[mu];            // y_mu (exact: s_mu is a power of two)
    acc = fmaf(yv, t * __half2float(q) / sL[mu], acc);
  }
  if (yy != nullptr) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float tot = 0.0f;
      for (int w = 0; w < 8; ++w) tot += red[w];
      yy[(size_t)b * n_yb] = tot;
      for (int i = 1; i < n_yb; ++i) yy[(size_t)b * n_yb + i] = 0.0f;
    }
  }
}

// ----------------------------------------------------------------------------
void launch_prepare_fp8(const double *src, int ld, int nr, int nc, const SysDev &s,
                        unsigned *colmax, uint8_t *L8, uint8_t *L8t, float *sL, cudaStream_t st) {
  cudaMemsetAsync(colmax, 0, sizeof(unsigned) * s.A, st);
  k_col_absmax<<<dim3((s.A + 31) / 32, (nr + 1023) / 1024), 256, 0, st>>>(src, ld, nr, nc,
                                                                         colmax);
  k_col_scales<<<(s.A + 255) / 256, 256, 0, st>>>(colmax, s.A, sL);
  k_quantize_L8<<<dim3((s.A + 31) / 32, (s.N + 31) / 32), 256, 0, st>>>(src, ld, nr, nc, s.N, s.A,
                                                                        sL, L8, L8t);
}

void launch_quant_x8(const __nv_bfloat16 *xh, int Bs, int N, uint8_t *x8, float *sx,
                     cudaStream_t st, const double *vscale) {
  k_quant_x8<<<Bs, 256, 0, st>>>(xh, Bs, N, x8, sx, vscale);
}

void launch_reduce_y_fp8(const float *Ypart, int splits, int Bs, int A, const float *sx,
                         const float *sL, uint8_t *y8, float *ty, float *yy, int n_yb,
                         cudaStream_t st) {
  k_reduce_y_fp8<<<Bs, 256, (size_t)A * sizeof(float), st>>>(Ypart, splits, Bs, A, sx, sL, y8, ty,
                                                             yy, n_yb);
}

void launch_quant_x16(const __nv_bfloat16 *xh, int Bs, int N, uint16_t *x16, float *sx,
                      cudaStream_t st, const double *vscale) {
  k_quant_x16<<<Bs, 256, 0, st>>>(xh, Bs, N, x16, sx, vscale);
}

void launch_reduce_y_f16(const float *Ypart, int splits, int Bs, int A, const float *sx,
                         const float *sL, uint16_t *y16, float *ty, float *yy, int n_yb,
                         cudaStream_t st) {
  k_reduce_y_f16<<<Bs, 256, (size_t)A * sizeof(float), st>>>(Ypart, splits, Bs, A, sx, sL, y16,
                                                             ty, yy, n_yb);
}

}  // namespace lgw
