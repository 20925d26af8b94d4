// Internal declarations of the lgw library (GB300, sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lgw.h"

namespace lgw {

// ---------------------------------------------------------------------------
// Layout constants
// ---------------------------------------------------------------------------
constexpr int PAD_VC = 128;    // pair dimension N_vc padded to a multiple of the GEMM2 M tile
constexpr int PAD_AUX = 128;   // N_aux padded to the GEMM1 M tile (also a multiple of the K block)
constexpr int PAD_VEC = 16;    // start vectors per sub-batch padded to the UMMA N granule
constexpr int VEC_THREADS = 256;
constexpr int VEC_E = 8;                             // pair elements per thread
constexpr int VEC_CHUNK = VEC_THREADS * VEC_E;       // pair elements per block
constexpr int F64_TILE = 64;                         // CUDA-core FP64 GEMM tile

// Device status bits (OR-ed into the handle's status word).
enum : unsigned {
  ST_NOT_SPD = 1u,
  ST_NO_CONV = 2u,
  ST_TIMEOUT = 4u,
  ST_BAD_INPUT = 8u,
};

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
inline int64_t round_up64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------------------
// Device-side system: padded copies owned by the system.
// ---------------------------------------------------------------------------
struct SysDev {
  int n_v, n_c, n_aux, n_vc;
  int N;        // n_vc padded to PAD_VC
  int A;        // n_aux padded to PAD_AUX
  double kf;    // c_K
  double *eps;      // [n_v + n_c]
  double *Delta;    // [N]  eps_c - eps_v, 0 in the padding
  double *dsq;      // [N]  Delta^1/2
  double *Delta2;   // [N]  Delta^2
  double *cd;       // [N]  c_K Delta^1/2
  float *dsqf;      // [N]  Delta^1/2 rounded to float (bf16 operand scaling)
  float *d2f;       // [N]  Delta^2 rounded to float   (alpha estimate)
  float *d2lo;      // [N]  Delta^2 - d2f rounded to float: (d2f, d2lo) is Delta^2 as a
                    //      double-float (the float-pair vector passes)
  float *cdf;       // [N]  c_K Delta^1/2 rounded to float (FP32 epilogue)
  double *L64;      // [N][A] row-major, zero padded
  __nv_bfloat16 *Lb;    // [N][A]   K-major operand of the L Y contraction
  __nv_bfloat16 *Ltb;   // [A][N]   operand of the L^T X contraction, K-block-major (kblk_bf16)
  __nv_bfloat16 *Lb_lo; // [N][A]   bf16(L - bf16(L)): second half of a split-BF16 L
  // E4M3 copies with power-of-two column scales, made on the first FP8 call
  uint8_t *L8;      // [N][A]   e4m3(L / s_mu)
  uint8_t *L8t;     // [A][N]   its transpose, K-block-major (kblk_e4m3)
  float *sL;        // [A]      s_mu
};

// ---------------------------------------------------------------------------
// One sub-batch of start vectors (Bs padded vectors, vector length N).
// ---------------------------------------------------------------------------
struct VecCtx {
  int N, Bs, nvec, nchunks;
  int k, kmax1;           // steps requested; k + 1
  int vec0;               // global index of the first vector of the sub-batch
  int reorth;             // lgw_reorth
  int ring;               // 1: FP64 vectors live in a 3-slot ring (slot j % 3)
  int nslots;             // FP64 slots (k + 1 for the FP64 basis, else 3)
  int slot0;              // without the ring, q_j lives in slot j - slot0 (a window of
                          // the basis, used by the recomputation from a checkpoint)
  int cpb;                // chunks per block of the assembly, axpy and normalisation
                          // passes (0 or 1: one; each chunk keeps its own partial)
  double tol;
  const double *Delta2, *dsq, *cd;
  double *w;              // [Bs][N]
  double *basis;          // slot s: basis + s * Bs * N
  __nv_bfloat16 *xh;      // [Bs][N]   bf16(Delta^1/2 q_j), K-block-major (kblk_bf16)
  float *bhi, *blo;       // split basis [k+1][Bs][N]: q = hi + lo (48 bits); blo may be
                          // null (float-only basis)
  const float *dsqf;      // [N]
  const float *d2f;       // [N] Delta^2 (float)
  const float *d2lo;      // [N] second float of Delta^2
  // pair: the ring slots and w hold float pairs (hi = the first Bs*N floats
  // of the slot, lo = the next Bs*N) and the vector passes run in double-
  // float arithmetic on the FP32 pipe (tensor-core path without
  // reorthogonalisation, ring mode)
  int pair;
  float2 *nalpha_f;       // [Bs] -alpha_j as a float pair (pair mode; written by the
                          // alpha reduction, so the passes convert no FP64 per thread)
  float2 *nbeta_f;        // [Bs] -beta_{j+1} as a float pair (pair mode; k_beta_vec)
  const float *ucd;       // [Bs][N] c_K Delta^1/2 (L y) from the FP32 epilogue (kblk_f32), or null
                          // (then w holds the full FP64 epilogue result)
  float *dq2_part;        // [Bs][nchunks] partials of sum Delta^2 q_j^2 (FP32); with
                          // LGW_REORTH_DCGS two halves by step parity, [2][Bs][nchunks]
  const float *yy_part;   // [Bs][n_yb]    partials of y . bf16(y) for the current q_j
  int n_yb;
  double kf;
  double *alpha_part;     // [n_mt][Bs]
  int n_mt;
  double *dot_part;       // [Bs][nchunks][kmax1]
  double *h;              // [Bs][kmax1]
  double *norm_a, *norm_b, *norm_c;   // [Bs][nchunks]
  int *flag2;             // [Bs] second CGS pass taken
  double *amax;           // [Bs]
  double *betaj;          // [Bs] beta_j for the running step
  double *sinv;           // [Bs] 1 / beta_{j+1} (0: stopped or not live), split path
  double *alpha, *beta, *beta0;   // global [B][k], [B][k], [B]
  int *k_eff;             // global [B]
  int *n_second;          // counter of second passes
  unsigned *status;
  // delayed Gram-Schmidt (LGW_REORTH_DCGS)
  double *wv;             // [Bs][N] the carried vector w_j (unnormalised q~_{j+1} = w_j / beta_{j+1})
  const double *uC;       // [Bs][N] C w_j from the FP64 contractions, or null (tensor cores)
  double *hj_part;        // [Bs][nchunks] partials of q_j . w_j
  double *gq;             // [Bs][kmax1] g = (T_{j-1} - alpha~_j) h / beta_j, removed by the sweep
};

// K-block-major layout of the GEMM1 operands (L^T and the per-step X):
// element (r, e) of a logical [rows][N] matrix (e along the contraction)
// sits at ((e / KB) * rows + r) * KB + e % KB, KB being one 128-byte row
// of the swizzled tile (64 BF16 or 128 E4M3 elements).  A TMA box of KB x
// box_rows is then one contiguous run of memory, so the contraction's
// concurrent tiles touch a handful of pages instead of one page per row
// (rows of a row-major [rows][1.6M] BF16 matrix are 3.2 MB apart).
// N must be a multiple of 128.
__host__ __device__ inline size_t kblk_bf16(int r, int e, int rows) {
  return ((size_t)(e >> 6) * rows + r) * 64 + (e & 63);
}
__host__ __device__ inline size_t kblk_e4m3(int r, int e, int rows) {
  return ((size_t)(e >> 7) * rows + r) * 128 + (e & 127);
}
// The FP32 contraction output ucd [Bs][N] (c_K Delta^1/2 L y, and the
// start-vector product V) in blocks of 128 pair elements: element (b, e) at
// ((e / 128) * Bs + b) * 128 + e % 128, so one 128 x BN output tile of the
// tensor-core epilogue is one contiguous run.
__host__ __device__ inline size_t kblk_f32(int b, int e, int Bs) {
  return ((size_t)(e >> 7) * Bs + b) * 128 + (e & 127);
}

__host__ __device__ inline double *slot_ptr(const VecCtx &c, int j) {
  int s = c.ring ? (j % 3) : (j - c.slot0);
  return c.basis + (size_t)s * c.Bs * c.N;
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in fixed order; every thread gets the result.  `red` needs
// blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// The same sum in the same order, formed by thread 0 only (the value is
// valid there alone): passes that only write a partial save the other
// threads' share of the final FP64 additions, which load GB300's narrow FP64
// pipe.
__device__ __forceinline__ double block_sum_to0(double v, double *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Transposed warp reduction of 32 values per lane: afterwards a[0] of lane l
// holds sum over all lanes of the original a[l].  31 shuffles per lane.
__device__ __forceinline__ void warp_transpose_sum32(double (&a)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      double send = up ? a[i] : a[i + off];
      double keep = up ? a[i + off] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
}

// Bounded device wait limit in clock cycles (about one second at 2 GHz).
constexpr long long WAIT_CYCLES = 2000000000LL;

// ---------------------------------------------------------------------------
// Host launchers (defined in the kernel files).  All take the stream last.
// ---------------------------------------------------------------------------
// k_prep.cu
void launch_pair_energies(const SysDev &s, cudaStream_t st);
void launch_pad_L(const double *L, const SysDev &s, cudaStream_t st);
void launch_quantize_L(const double *src, int ld, int nr, int nc, const SysDev &s,
                       cudaStream_t st);
void launch_check_delta(const SysDev &s, unsigned *status, cudaStream_t st);

// k_gemm_f64.cu : CUDA-core FP64 contractions
// Ypart[split][Bs][A] = sum_vc (Delta^1/2 q)[b][vc] L[vc][mu] over the split's vc range
int gemm1_f64_splits(const SysDev &s, int Bs);
void launch_gemm1_f64(const SysDev &s, const double *q, int Bs, double *Ypart, int splits,
                      cudaStream_t st);
void launch_reduce_y_f64(const double *Ypart, int splits, int Bs, int A, double *Y, cudaStream_t st);
// U[b][vc] = sum_mu Y[b][mu] L[vc][mu]; epilogue:
//   EPI_START:   w = Delta^1/2 U
//   EPI_LANCZOS: w = Delta^2 q + c_K Delta^1/2 U - beta_j q_prev; alpha partials per 64-row tile
//   EPI_APPLY:   w = C q = Delta^2 q + c_K Delta^1/2 U; q . w partials per tile if alpha_part
enum { EPI_START = 0, EPI_LANCZOS = 1, EPI_APPLY = 2 };
void launch_gemm2_f64(const SysDev &s, const double *Y, int Bs, int epi, const double *q,
                      const double *qprev, const double *betaj, double *w, double *alpha_part,
                      cudaStream_t st);

// k_gemm_tc.cu : BF16 tcgen05 contractions
struct TcPlan;
bool tc_available();
bool tc_plan_enable_fp8(TcPlan *p, const uint8_t *L8t, const uint8_t *L8, const uint8_t *x8,
                        const uint8_t *y8, const float *ty);
void launch_prepare_fp8(const double *src, int ld, int nr, int nc, const SysDev &s,
                        unsigned *colmax, uint8_t *L8, uint8_t *L8t, float *sL, cudaStream_t st);
// vscale (optional, [Bs]): normalisation factor of an unnormalised operand,
// folded into sx
void launch_quant_x8(const __nv_bfloat16 *xh, int Bs, int N, uint8_t *x8, float *sx,
                     cudaStream_t st, const double *vscale = nullptr);
void launch_reduce_y_fp8(const float *Ypart, int splits, int Bs, int A, const float *sx,
                         const float *sL, uint8_t *y8, float *ty, float *yy, int n_yb,
                         cudaStream_t st);
// E4M3 L widened to FP16 in shared memory (precision LGW_FP8_DEQ): the
// per-step operands in FP16 with per-vector power-of-two scales.
bool tc_plan_enable_deq(TcPlan *p, const uint8_t *L8t, const uint8_t *L8, const uint16_t *x16,
                        const uint16_t *y16, const float *ty);
void launch_quant_x16(const __nv_bfloat16 *xh, int Bs, int N, uint16_t *x16, float *sx,
                      cudaStream_t st, const double *vscale = nullptr);
void launch_reduce_y_f16(const float *Ypart, int splits, int Bs, int A, const float *sx,
                         const float *sL, uint16_t *y16, float *ty, float *yy, int n_yb,
                         cudaStream_t st);
bool tc_plan_has_bf16(const TcPlan *p);
bool tc_plan_autotune(TcPlan *p, float *ucd, unsigned *status, cudaStream_t st, int *splits_out);
TcPlan *tc_plan_create(const SysDev &s, int Bs, const __nv_bfloat16 *xh, float *ypart,
                       __nv_bfloat16 *yh, int *splits_out, char *err, size_t errn);
void tc_plan_destroy(TcPlan *p);
void launch_gemm1_tc(const TcPlan *p, unsigned *status, cudaStream_t st);
// Yh = bf16(sum of split partials); yy (optional, [Bs][A/256]) receives
// per-block partials of sum_mu y_mu * Yh_mu for the alpha estimate.
// vscale (optional, [Bs]) multiplies each vector's sum before rounding: the
// normalisation of an operand that was contracted unnormalised.
void launch_reduce_y_bf16(const float *Ypart, int splits, int Bs, int A, __nv_bfloat16 *Yh,
                          float *yy, cudaStream_t st, const double *vscale = nullptr);
void launch_gemm2_tc(const TcPlan *p, int epi, const double *q, const double *qprev,
                     const double *betaj, double *w, double *alpha_part, unsigned *status,
                     cudaStream_t st);
// Store-only FP32 epilogue for the split basis: ucd = c_K Delta^1/2 U.
void launch_gemm2_tc_split(const TcPlan *p, float *ucd, unsigned *status, cudaStream_t st);
// Coupling vectors V = L M in split BF16 on the tensor cores:
// V ~ L_hi M_hi + L_hi M_lo + L_lo M_hi (FP32 accumulation into vf [Bs][N]).
// M rows [nvec][n_aux] (FP64, device); uses the plan's yh buffer for the
// bf16 halves of M.
bool launch_coupling_tc(const TcPlan *p, const SysDev &s, const double *M, int nvec,
                        float *vf, unsigned *status, cudaStream_t st);
int tc_n_mt(const SysDev &s);
// one block: a bounded wait of limit_cycles on a barrier that is completed
// (arrive != 0) or never completed (ST_TIMEOUT)
void launch_wait_selftest(int arrive, long long limit_cycles, unsigned *status, cudaStream_t st);

// k_lanczos.cu : vector kernels of one step
void launch_start_from_v(const VecCtx &c, const double *V, int ldv, int n_valid, cudaStream_t st);
// w = Delta^1/2 vf (vf float [Bs][N], rows >= nvec ignored) and ||w||^2 partials.
void launch_start_from_vf(const VecCtx &c, const float *vf, cudaStream_t st);
void launch_norm_partials(const VecCtx &c, const double *x, double *out, cudaStream_t st);
void launch_normalize(const VecCtx &c, int j, int is_start, const double *norm, cudaStream_t st);
void launch_assemble_w(const VecCtx &c, int j, const float *ucd, cudaStream_t st);
void launch_alpha_reduce(const VecCtx &c, int j, cudaStream_t st);
void launch_alpha_axpy(const VecCtx &c, int j, cudaStream_t st);
void launch_beta_vec(const VecCtx &c, int j, cudaStream_t st);
void launch_reduce_dots(const VecCtx &c, int j, int pass, cudaStream_t st);
void launch_update(const VecCtx &c, int j, int pass, cudaStream_t st);
void launch_dots(const VecCtx &c, int j, int pass, cudaStream_t st);
void launch_second_pass_decide_j(const VecCtx &c, int j, cudaStream_t st);
// Band Lanczos (off-diagonal Sigma_tt'): one recurrence per group (a summed
// orbital) whose start block holds the p targets' vectors; one new basis
// vector per step, CGS2 against all of the group's vectors, FP64 basis.
struct BandCtx {
  VecCtx c;          // groups as the sub-batch's vectors: basis (ring 0), w, xh,
                     // dot_part, h, norm_a/b/c, vec0, nvec, k, kmax1, tol
  int p;             // band width (targets)
  int G;             // groups of the whole request
  int *nv;           // [Bs] basis vectors formed
  int *act;          // [Bs] the group takes part in the current operation
  int *newrow;       // [Bs] row the current operation appends, or -1
  double *inv;       // [Bs] 1 / norm of the appended vector
  double *hsum;      // [Bs][kmax1] projection coefficients of both passes
  double *scale;     // [Bs] largest start-vector norm (breakdown scale of the start)
  double *tmax;      // [Bs] largest |T| entry so far (breakdown scale of the steps)
  double *Tb;        // [G][k][p+1] Tb[g][j][d] = T[j+d][j]
  double *R0;        // [G][p][p]   b_a = sum_i R0[g][i][a] q_i
  int *keff;         // [G]         steps (columns of T) taken
  double *xq;        // [Bs][N] FP64 operand for the FP64 contractions, or null
};
void launch_band_init(const BandCtx &bc, cudaStream_t st);
void launch_band_activate(const BandCtx &bc, int mode, int j, cudaStream_t st);
void launch_band_operand(const BandCtx &bc, int j, cudaStream_t st);
void launch_band_assemble(const BandCtx &bc, int j, const float *ucd, cudaStream_t st);
// one orthogonalise-and-append: CGS2 of w against the group's vectors, the
// coefficient record (mode 0: column idx of R0; mode 1: column idx of T),
// breakdown test and the new basis vector
// the new basis vector; returns the number of kernels launched
int launch_band_append(const BandCtx &bc, int mode, int idx, cudaStream_t st);
void launch_band_finish(const BandCtx &bc, cudaStream_t st);
// Lanczos on each group's small banded T from y = R0 x for the nx
// polarisation vectors x [nx][p]; output tridiagonals [nx * G][k] (vector
// index xi * G + g); scratch: nx * G * (k + 2) * k doubles
void launch_band_small(const double *Tb, const double *R0, const int *keff, int G, int k, int p,
                       const double *xs, int nx, double tol, double *scratch, double *alpha,
                       double *beta, double *beta0, int *keff_out, cudaStream_t st);
// out [p][p][F][2] from the nx fraction sums sig [nx][F][2]: diagonal a from
// x = a, pair (a, b) from (x+ - x-) / 4
void launch_band_combine(const double *sig, int p, int F, double *out, cudaStream_t st);

// k_reorth.cu : split-precision basis (double-float dots, FP32 small updates)
void launch_dots_split(const VecCtx &c, int j, int pass, cudaStream_t st);
void launch_reduce_dots_split(const VecCtx &c, int j, int pass, cudaStream_t st);
void launch_update_split(const VecCtx &c, int j, int pass, cudaStream_t st);
void launch_start_split(const VecCtx &c, cudaStream_t st);
// delayed Gram-Schmidt: one sweep over the basis per step, its per-vector
// reduction, and the second pass of the vectors the reduction flags
void launch_sweep_dcgs(const VecCtx &c, int j, cudaStream_t st);
void launch_reduce_dcgs(const VecCtx &c, int j, cudaStream_t st);
void launch_pass2_dcgs(const VecCtx &c, int j, cudaStream_t st);
void launch_scale_rows_to_bf16(const double *x, const double *dsq, int Bs, int N,
                               __nv_bfloat16 *out, cudaStream_t st);

// k_spectral.cu : tridiagonal -> Gauss rule -> Omega-space Jacobi matrix
struct JacobiBufs {
  double *a;    // [B][k]
  double *b2;   // [B][k]  b2[i][j] = b_{j+1}^2 couples j and j+1
  double *w0;   // [B]     total weight (zeroth moment)
  int *n;       // [B]     depth
  // polynomial variant: G(0) per vector, and the fractions belong to
  // D = p_g(C) (Sigma_tm = (G(zeta) - G(0)) / z); NULL for the Omega-space
  // fractions of the spectral map (Sigma_tm = -eta G(zeta))
  double *g0 = nullptr;
};

// k_poly.cu : one vector pass of Clenshaw's recurrence for p_g(C) q
struct PolyStep {
  int N;
  const double *q;        // [Bs][N] the Lanczos vector q_j
  const double *b1, *b2;  // b_{k+1}, b_{k+2} or NULL
  const double *T;        // C b1 in FP64, or NULL
  const float *ucd;       // c_K Delta^1/2 (L y) of b1 in FP32 (with T == NULL)
  const double *Delta2;
  const float *dsqf;
  double ck, as, bs;      // c_k, a_s, b_s
  double *out;            // b_k
  __nv_bfloat16 *xh;      // bf16(Delta^1/2 b_k) or NULL
};
void launch_cheb_step(const PolyStep &p, int nchunks, int Bs, cudaStream_t st);
void launch_cheb_final(const PolyStep &p, const double *qprev, const double *betaj, double *w,
                       double *alpha_part, int nchunks, int Bs, cudaStream_t st);
void launch_poly_prep(const double *alpha, const double *beta, const double *beta0,
                      const int *k_eff, int B, int k, JacobiBufs jb, unsigned *status,
                      cudaStream_t st);
// scratch: 3 * B * k doubles; min_theta_bits: running minimum of the Gauss
// nodes (positive doubles compare like their bit patterns)
void launch_spectral_impl(const double *alpha, const double *beta, const double *beta0,
                          const int *k_eff, int B, int k, JacobiBufs jb, double *scratch,
                          unsigned long long *min_theta_bits, unsigned *status, cudaStream_t st);

// make_vector: a hash start vector vec [N] (entries in [-1, 1), zero
// padding); otherwise out[0..1] = [min Delta^2, largest Ritz value of the
// tridiagonal (a, b) of depth *k_eff plus its last off-diagonal]
void launch_interval(const double *Delta2, int n_vc, int N, const double *a, const double *b,
                     const int *k_eff, double *out, double *vec, unsigned long long seed,
                     bool make_vector, cudaStream_t st);

// k_cf.cu : continued fractions on the grid and QP solve
struct CfProblem {
  int n_t, n_m, n_freq, k;
  const int *targets, *m_idx;   // device
  const double *eps;            // device [n_v + n_c]
  int n_v;
  const double *omega;          // device [n_freq]
  double delta;
  const double *shift;          // device [n_t] or nullptr
  int qp_mode;                  // 0 graphical (Newton), 1 linearised at eps_t + s_t
};
int cf_slices(const CfProblem &p);
// part: S * n_t * n_freq * 2 doubles of scratch, or NULL for one slice;
// returns the number of kernels launched
int launch_cf_grid(const CfProblem &p, JacobiBufs jb, double *sigma, double *part, int S,
                   cudaStream_t st);
void launch_qp(const CfProblem &p, JacobiBufs jb, const double *sigma, int max_iter, double tol,
               double *e_qp, double *z_qp, unsigned *status, cudaStream_t st);

void launch_tda_view(const double *Delta, int n_vc, int N, double c, double *ones, double *cd,
                     float *onesf, float *d2f, float *d2lo, float *cdf, cudaStream_t st);
void launch_pol_rows(const double *src, int n_m, int len, const int *pairs, int n_pairs,
                     double *dst, cudaStream_t st);
void launch_pol_combine(const double *sig2, int n_pairs, int n_freq, double *out,
                        cudaStream_t st);

// k_static.cu : exchange self-energy and density-fitting factors
void launch_sigma_x(const double *M, int n_t, int n_m, int n_aux, const int *m_idx, int n_v,
                    double *out, cudaStream_t st);
int launch_cholesky(double *A, int n, unsigned *status, cudaStream_t st);
void launch_gemm_nn_f64(const double *A, const double *B, int M, int N, int K, double *C,
                        cudaStream_t st);

// k_adjoint.cu : gradient of the QP energies (implicit function + Daleckii-Krein)
// A stored Krylov basis [slot][Bs][N]: FP64, or the float pair hi (+ lo).
struct BasisRef {
  const double *d;
  const float *hi, *lo;
  __device__ __forceinline__ double at(size_t i) const {
    if (d) return d[i];
    return lo ? (double)hi[i] + (double)lo[i] : (double)hi[i];
  }
};
struct AdjCtx {
  int N, Bs, nvec, vec0, k, n_m, n_v;
  const double *alpha, *beta, *beta0;   // [B][k], [B][k], [B]
  const int *k_eff;                     // [B]
  const double *E, *Z, *dE;             // [n_t]
  const double *eps;                    // [n_v + n_c]
  const int *m_idx;                     // [n_m]
  double delta;
  double *theta;   // [Bs][k]
  double *V;       // [Bs][k][k]  V[s][i]: component i of eigenvector s of T_k
  double *Phi;     // [Bs][k][k]
  double *X;       // [Bs][k][k]  U Phi
  double *ay;      // [Bs][k]
  double *Gam;     // [Bs][k][k]
  float *Gamf;     // [Bs][k][k] FP32 copy of Gam, or NULL
  double *dz;      // [Bs]
  unsigned *status;
  // Tamm-Dancoff: F = b^T (z + eta A)^-1 b with A = Delta + c L L^T and
  // b = L M (the nodes are theta, not Omega = sqrt(theta); A is linear in
  // Delta and b does not depend on it)
  int tda;
  // polynomial form: the nodes of D = p_g(C)'s tridiagonal are Omega
  // directly, f(Omega) = 1 / (Omega (z + eta Omega))
  int poly;
};
// Reverse mode of the three-term recurrence (no reorthogonalisation) over
// one segment of steps [s0, e) of a sub-batch, the steps taken back from
// e - 1 to s0.  Vector buffers are [Bs][N] per slot.
struct RevCtx {
  int N, Bs, nvec, vec0, k, nchunks;
  int s0;                 // first step of the segment
  const double *seg;      // q_{s0-1} .. q_e at slot j - s0 + 1 (q_{-1} = 0)
  double *qbar;           // [3] adjoints of q_j at slot j % 3
  const double *cu;       // C ubar_{j+1} of the step taken back before (0 at the start)
  double *useg;           // ubar_j at slot j - s0
  double *Gd;             // [Bs][N] running diag(dF/dC): sum_j ubar_j o q_j when the
                          // recurrence runs on C (gd_from_steps), else added by the caller
  int gd_from_steps;
  double *dpart;          // [Bs][nchunks][6] dot-product partials
  double *coef;           // [Bs][8] per-vector coefficients of the running step
  double *bbar;           // [Bs][k] running adjoints of beta[j] (coupling of j, j+1)
  const double *Gam;      // [Bs][k][k] dF/dT_k (weights folded in)
  const double *ay;       // [Bs][k]; ay[0] = dF/dbeta0
  const double *alpha, *beta, *beta0;   // global [B][k], [B][k], [B]
  const int *k_eff;       // global [B]
};
void launch_rev_init(const RevCtx &r, cudaStream_t st);
void launch_rev_set_betaj(const RevCtx &r, double *betaj, cudaStream_t st);
void launch_rev_step(const RevCtx &r, int j, cudaStream_t st);
void launch_rev_finish(const RevCtx &r, const double *q0, double *Y, cudaStream_t st);
void launch_rev_axpby(double *out, double a, const double *x, double b, size_t n,
                      cudaStream_t st);
void launch_rev_gd(double *Gd, double coef, const double *x, const double *y, size_t n,
                   cudaStream_t st);
int adj_max_k();
bool tc_gemm_f64out(int np, const __nv_bfloat16 *const *A, const int *a_kblk,
                    const __nv_bfloat16 *const *B, int M, int Ncols, int K, int kchunk,
                    double *out, int ldo, int add, unsigned *status, cudaStream_t st, char *err,
                    size_t errn);
void launch_split_t(BasisRef src, int R, int C, int lds, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                    cudaStream_t st);
void launch_split_scaled(BasisRef src, int R, int C, const double *scale, __nv_bfloat16 *hi,
                         __nv_bfloat16 *lo, cudaStream_t st);
void launch_adj_rows_f32(const AdjCtx &a, BasisRef basis, double *Y, double *Gd,
                         cudaStream_t st);
void launch_eig_full(const AdjCtx &a, cudaStream_t st);
void launch_adj_coeffs(const AdjCtx &a, cudaStream_t st);
void launch_adj_rows(const AdjCtx &a, BasisRef basis, double *Y, double *Gd, cudaStream_t st);
void launch_gamma_p(const AdjCtx &a, const double *P, int A, double *R, cudaStream_t st);
// S[i][mu] += scale * sum_r X[r][i] Yr[r][mu]
void launch_atb_f64(const double *X, int ldx, const double *Yr, int ldy, int R, int Ni, int Nmu,
                    double *S, cudaStream_t st, double scale = 1.0);
void launch_adj_accumulate(const AdjCtx &a, const double *Delta, BasisRef basis,
                           const double *Y, const double *Gd, double *dDelta, double *deps,
                           cudaStream_t st);
void launch_adj_dL(const double *L64, const double *dsq, const double *SC, const double *SB,
                   int A, int n_vc, int n_aux, double kf, double *dL, double *dDelta, int tda,
                   cudaStream_t st);
void launch_adj_deps(const double *dDelta, int n_v, int n_c, const int *targets, int n_t,
                     const double *Z, const double *dE, double *deps, cudaStream_t st);

}  // namespace lgw
