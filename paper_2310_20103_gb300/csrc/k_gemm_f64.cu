// CUDA-core FP64 contractions of the low-rank Casida matvec.
//
// C x = Delta^2 x + c_K Delta^1/2 L (L^T (Delta^1/2 x))   (Eq. 4 with K = L L^T)
//
// gemm1: Y = L^T (Delta^1/2 X), split over the pair dimension (long K).
// gemm2: U = L Y with the Lanczos epilogue w = Delta^2 q + c_K Delta^1/2 U -
//        beta_j q_{j-1} and per-tile partial sums of alpha_j = q_j . w.
// These run on the FP64 pipe (about 1.2 TFLOP/s on GB300); they are the
// plain FP64 path and the FP64 coupling-vector product V = L M.
#include "lgw_internal.cuh"

namespace lgw {

constexpr int TB = F64_TILE;   // 64 x 64 output tile
constexpr int BK = 16;

__global__ void __launch_bounds__(256) k_gemm1_f64(const double *__restrict__ L64,
                                                   const double *__restrict__ dsq,
                                                   const double *__restrict__ q, int N, int A,
                                                   int Bs, int kb_per_split,
                                                   double *__restrict__ Ypart) {
  __shared__ double As[BK][TB + 1];
  __shared__ double Bt[BK][TB + 1];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int mu0 = blockIdx.x * TB, b0 = blockIdx.y * TB, split = blockIdx.z;
  const int nkb = N / BK;
  const int kb_lo = split * kb_per_split;
  const int kb_hi = min(nkb, kb_lo + kb_per_split);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int kb = kb_lo; kb < kb_hi; ++kb) {
    const int vc0 = kb * BK;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = t + 256 * r;
      int kk = idx & 15, m = idx >> 4;
      int b = b0 + m;
      As[kk][m] = (b < Bs) ? dsq[vc0 + kk] * q[(size_t)b * N + vc0 + kk] : 0.0;
      int n = idx & 63, k2 = idx >> 6;
      Bt[k2][n] = L64[(size_t)(vc0 + k2) * A + mu0 + n];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bt[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double *out = Ypart + (size_t)split * Bs * A;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int b = b0 + ty + 16 * i;
    if (b >= Bs) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(size_t)b * A + mu0 + tx + 16 * j] = acc[i][j];
  }
}

__global__ void k_reduce_y_f64(const double *__restrict__ Ypart, int splits, int n,
                               double *__restrict__ Y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int p = 0; p < splits; ++p) s += Ypart[(size_t)p * n + i];
  Y[i] = s;
}

__global__ void __launch_bounds__(256) k_gemm2_f64(const double *__restrict__ L64,
                                                   const double *__restrict__ Y, int N, int A,
                                                   int Bs, int epi,
                                                   const double *__restrict__ Delta2,
                                                   const double *__restrict__ dsq,
                                                   const double *__restrict__ cd,
                                                   const double *__restrict__ q,
                                                   const double *__restrict__ qprev,
                                                   const double *__restrict__ betaj,
                                                   double *__restrict__ w,
                                                   double *__restrict__ alpha_part) {
  __shared__ double As[BK][TB + 1];
  __shared__ double Bt[BK][TB + 1];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int vc0 = blockIdx.x * TB, b0 = blockIdx.y * TB;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int mu0 = 0; mu0 < A; mu0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = t + 256 * r;
      int kk = idx & 15, m = idx >> 4;
      int b = b0 + m;
      As[kk][m] = (b < Bs) ? Y[(size_t)b * A + mu0 + kk] : 0.0;
      Bt[kk][m] = L64[(size_t)(vc0 + m) * A + mu0 + kk];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bt[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int b = b0 + ty + 16 * i;
    const bool bok = b < Bs;
    double apart = 0.0;
    const double bj = (epi == EPI_LANCZOS && bok && betaj != nullptr) ? betaj[b] : 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int vc = vc0 + tx + 16 * j;
      if (!bok) continue;
      const size_t o = (size_t)b * N + vc;
      if (epi == EPI_START) {
        w[o] = dsq[vc] * acc[i][j];
      } else {
        const double qv = q[o];
        double wv = fma(Delta2[vc], qv, cd[vc] * acc[i][j]);
        if (epi == EPI_LANCZOS && qprev != nullptr) wv = fma(-bj, qprev[o], wv);
        w[o] = wv;
        apart = fma(qv, wv, apart);
      }
    }
    if ((epi == EPI_LANCZOS || epi == EPI_APPLY) && alpha_part != nullptr) {
      // sum over the 16 threads (tx) that share row b: lanes differ in bits 0..3
#pragma unroll
      for (int o = 8; o >= 1; o >>= 1) apart += __shfl_xor_sync(0xffffffffu, apart, o);
      if (tx == 0 && bok) alpha_part[(size_t)blockIdx.x * Bs + b] = apart;
    }
  }
}

int gemm1_f64_splits(const SysDev &s, int Bs) {
  int tiles = (s.A / TB) * ((Bs + TB - 1) / TB);
  int nkb = s.N / BK;
  int splits = (304 + tiles - 1) / tiles;
  int maxs = nkb / 8 > 0 ? nkb / 8 : 1;
  if (splits > maxs) splits = maxs;
  if (splits < 1) splits = 1;
  int per = (nkb + splits - 1) / splits;
  return (nkb + per - 1) / per;
}

void launch_gemm1_f64(const SysDev &s, const double *q, int Bs, double *Ypart, int splits,
                      cudaStream_t st) {
  int nkb = s.N / BK;
  int per = (nkb + splits - 1) / splits;
  dim3 grid(s.A / TB, (Bs + TB - 1) / TB, splits);
  k_gemm1_f64<<<grid, 256, 0, st>>>(s.L64, s.dsq, q, s.N, s.A, Bs, per, Ypart);
}

void launch_reduce_y_f64(const double *Ypart, int splits, int Bs, int A, double *Y,
                         cudaStream_t st) {
  int n = Bs * A, th = 256;
  k_reduce_y_f64<<<(n + th - 1) / th, th, 0, st>>>(Ypart, splits, n, Y);
}

void launch_gemm2_f64(const SysDev &s, const double *Y, int Bs, int epi, const double *q,
                      const double *qprev, const double *betaj, double *w, double *alpha_part,
                      cudaStream_t st) {
  dim3 grid(s.N / TB, (Bs + TB - 1) / TB);
  k_gemm2_f64<<<grid, 256, 0, st>>>(s.L64, Y, s.N, s.A, Bs, epi, s.Delta2, s.dsq, s.cd, q, qprev,
                                    betaj, w, alpha_part);
}

}  // namespace lgw
