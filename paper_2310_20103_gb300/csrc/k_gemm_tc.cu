// BF16 tensor-core contractions of the low-rank Casida matvec on sm_103a:
// tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 accumulator in tensor memory),
// operands staged by TMA (cp.async.bulk.tensor, 128-byte swizzle), a
// multi-stage mbarrier pipeline, and the epilogue read back with tcgen05.ld.
//
//   gemm1: Y^T[mu][b] = sum_vc L^T[mu][vc] Xh[b][vc]     (M = N_aux, K = N_vc)
//          Xh = bf16(Delta^1/2 q_j) (written by the normalisation kernel);
//          split over K, FP32 partials reduced in fixed order into bf16 Yh.
//   gemm2: U[vc][b] = sum_mu L[vc][mu] Yh[b][mu]          (M = N_vc, K = N_aux)
//          fused FP64 epilogue w = Delta^2 q_j + c_K Delta^1/2 U - beta_j q_{j-1}
//          and per-tile partial sums of alpha_j = q_j . w (warp-transposed
//          reduction, fixed-order sum over the four epilogue warps).
//
// Both operands are K-major (row-major with K contiguous): L^T [N_aux][N_vc]
// for gemm1 and L [N_vc][N_aux] for gemm2, so each gemm has its own copy.
// CTA = 6 warps: warp 0 issues TMA, warp 1 owns tensor memory and issues the
// MMAs from one thread, warps 2..5 run the epilogue (warp w reads TMEM lanes
// 32*(w%4) .. 32*(w%4)+31).  Tile 128 x BN x 64, BN in {64, 128, 256}.
// Every mbarrier wait is bounded (clock64); a timeout sets ST_TIMEOUT.
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>

#include "lgw_internal.cuh"

namespace lgw {
namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;              // 64 bf16 = 128 bytes = one swizzle row
constexpr int NTHREADS = 192;

// HALF: half the pipeline stages (about 100 KB of shared memory), so that
// two CTAs fit on an SM and one's epilogue overlaps the other's main loop
// (tensor memory: 2 x BN <= 512 columns).  Used for the store-only
// contraction, whose K loop is short.
// DEQ: the A operand arrives as E4M3 (RAW_BYTES per stage, 64 bytes by 128
// rows) next to the B tile, and is widened to FP16 into a ring of its own
// (A_SLOTS tiles ahead of the TMA stages), so the TMA ring stays as deep as
// the BF16 one while the conversion runs one K block ahead of the MMAs.
template <int BN, int HALF = 0, bool DEQ = false>
struct Cfg {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int RAW_BYTES = DEQ ? BM * BK : 0;
  static constexpr int A_SLOTS = DEQ ? 2 : 0;
  static constexpr int A_RING = A_SLOTS * A_BYTES;
  static constexpr int B_OFF = DEQ ? 0 : A_BYTES;   // B tile within a stage
  static constexpr int RAW_OFF = B_OFF + B_BYTES;
  static constexpr int STAGE = (DEQ ? 0 : A_BYTES) + B_BYTES + RAW_BYTES;
  static constexpr int STAGES =
      DEQ ? (BN == 256 ? 4 : (BN == 128 ? 6 : 8))
          : (((BN == 256) ? 4 : (BN == 128 ? 6 : 8)) >> HALF);
  static constexpr int BAR_BYTES = 256;
  static constexpr int RED_BYTES = 4 * BN * 8;
  static constexpr int SMEM = 1024 + A_RING + STAGES * STAGE + BAR_BYTES + RED_BYTES;
  static constexpr uint32_t TMEM_COLS = BN;
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait on a barrier phase: false (and ST_TIMEOUT in *status) once
// `limit` clock cycles have passed without the phase completing.
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t parity, unsigned *status,
                                              long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > limit) {
      atomicOr(status, ST_TIMEOUT);
      return false;
    }
  }
}
// The pipeline's waits: ~1 s.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *status) {
  return mbar_wait_for(bar, parity, status, WAIT_CYCLES);
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, uint64_t *bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// 3-D form for the K-block-major operands: (0, row, K block)
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, uint64_t *bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem desc] * B[smem desc]^T, M=128, N=BN, K=16 (bf16)
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// D[tmem] (+)= A * B^T, M=128, N=BN, K=32 (E4M3 x E4M3, FP32 accumulator)
__device__ __forceinline__ void umma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on an mbarrier once every MMA issued so far by this thread is done.
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO); LBO unused for this layout.
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address  [0,14)
  d |= (uint64_t)1 << 16;                     // LBO (16 B)      [16,30)
  d |= (uint64_t)(1024 >> 4) << 32;           // SBO             [32,46)
  d |= (uint64_t)1 << 46;                     // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                     // swizzle mode: 128-byte
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor, kind::f8f6f4: FP32 accumulator, A and B E4M3
// (format code 0), both K-major.
__host__ __device__ constexpr uint32_t make_idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor, kind::f16 with FP16 A and B (format code 0): the
// widened E4M3 operand and its FP16 partner.
__host__ __device__ constexpr uint32_t make_idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Orders this thread's generic-proxy shared-memory writes before later
// reads by the tensor cores (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// E4M3 -> FP16 is exact for every E4M3 value, subnormals included.
// One instruction per pair: the lower byte of each 16-bit half is the first
// element and lands in the lower FP16 half.
__device__ __forceinline__ uint32_t cvt_e4m3x2_f16x2(uint32_t pair16) {
  uint32_t d;
  asm("{\n\t.reg .b16 a;\n\tcvt.u16.u32 a, %1;\n\tcvt.rn.f16x2.e4m3x2 %0, a;\n\t}"
      : "=r"(d)
      : "r"(pair16));
  return d;
}

struct EpiArgs {
  // gemm1 (split-K partials)
  float *ypart;          // [splits][ncols][ldo]
  int ldo;
  // gemm2 (Lanczos epilogue)
  int N;                 // vector length
  const double *Delta2, *cd, *q, *qprev, *betaj;
  double *w, *alpha_part;
  unsigned *status;
  // split-basis epilogue (FP32)
  const float *qh, *qph, *d2f, *cdf;
  float *ucd;
  // FP64 output (E_F64): out[col * ldo + row] (=, or += when add != 0)
  double *out;
  int add;
  // per-column (vector) scale of the accumulator (FP8 operands), or NULL
  const float *colscale;
  // K loop start rotated by the M tile (spreads concurrent CTAs over HBM
  // channels) or not (CTAs sharing the B tile stream it in step, from L2)
  int rot;
  // operand maps are 3-D K-block-major (kblk_*) instead of 2-D row-major
  int a3, b3;
  // tile numbering in launch order: 0 = N tiles fastest (CTAs sharing an L
  // tile run together), 1 = M tiles fastest (CTAs sharing the B tile run
  // together)
  int mfast;
};

enum { E_SPLITK = 0, E_LANCZOS = 1, E_APPLY = 2, E_LANCZOS_NA = 3, E_SPLITB = 4, E_VACC = 5,
       E_F64 = 6 };

// EB: operand element bytes, 2 = BF16 (kind::f16, K block 64), 1 = E4M3
// (kind::f8f6f4, K block 128); a K block is one 128-byte swizzle row either way.
// EB = 3: E4M3 A operand widened to FP16 in shared memory by the four
// epilogue warps during the main loop, FP16 B operand (kind::f16, K block 64).
template <int BN, int EPI, int EB, int HALF = 0>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int M, int Ncols, int num_kb, int kb_per_split, EpiArgs ea) {
  constexpr bool DEQ = EB == 3;
  using C = Cfg<BN, HALF, DEQ>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t *aring = smem;                 // DEQ: widened A tiles
  uint8_t *stages = smem + C::A_RING;
  uint64_t *full = reinterpret_cast<uint64_t *>(stages + C::STAGES * C::STAGE);
  uint64_t *empty = full + C::STAGES;
  uint64_t *conv = empty + C::STAGES;    // DEQ: A slot widened (4 warps)
  uint64_t *afree = conv + C::A_SLOTS;   // DEQ: A slot read by the MMAs
  uint64_t *tfull = afree + C::A_SLOTS;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(tfull + 1);
  double *red = reinterpret_cast<double *>(smem + C::STAGES * C::STAGE + C::BAR_BYTES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // CTAs are dispatched in linear block order (x fastest).  Numbering the
  // tiles of that order with N fastest makes the CTAs that share an L tile
  // (all N tiles of one M tile) run together, so L streams from HBM once
  // and its other reads hit L2; M fastest instead keeps the CTAs of one B
  // tile together (chosen per shape by the autotuner).  With rotation each
  // M tile starts its K loop at a different block, spreading concurrent
  // requests over HBM channels; CTAs of one M tile keep the same start.
  const int n_tiles = gridDim.y;
  const int lin = blockIdx.x + blockIdx.y * gridDim.x;
  const int m_tile = ea.mfast ? (int)blockIdx.x : lin / n_tiles;
  const int n_tile = ea.mfast ? (int)blockIdx.y : lin % n_tiles;
  const int split = blockIdx.z;
  const int kb0 = split * kb_per_split;
  const int kb1 = min(num_kb, kb0 + kb_per_split);
  const int nk = max(0, kb1 - kb0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < C::A_SLOTS; ++a) {
      mbar_init(&conv[a], 4);   // one arrival per converting warp
      mbar_init(&afree[a], 1);
    }
    mbar_init(tfull, 1);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tslot, C::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nk; ++it) {
        const int s = it % C::STAGES;
        const uint32_t ph = (it / C::STAGES) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, ea.status)) break;
        mbar_expect_tx(&full[s], C::STAGE);
        uint8_t *sa = stages + s * C::STAGE;
        const int kb = kb0 + (it + (ea.rot ? m_tile : 0)) % nk;
        const int kx = kb * (EB == 1 ? 128 : 64);
        if (DEQ) {
          // E4M3 A: half of a 128-element K block (K-block-major) or the
          // 64 columns kx.. of a row-major operand; 64 bytes by 128 rows
          uint8_t *raw = sa + C::RAW_OFF;
          if (ea.a3)
            tma_load_3d(raw, &tmA, &full[s], (kb & 1) * 64, m_tile * BM, kb >> 1);
          else
            tma_load_2d(raw, &tmA, &full[s], kx, m_tile * BM);
        } else if (ea.a3) {
          tma_load_3d(sa, &tmA, &full[s], 0, m_tile * BM, kb);
        } else {
          tma_load_2d(sa, &tmA, &full[s], kx, m_tile * BM);
        }
        if (ea.b3)
          tma_load_3d(sa + C::B_OFF, &tmB, &full[s], 0, n_tile * BN, kb);
        else
          tma_load_2d(sa + C::B_OFF, &tmB, &full[s], kx, n_tile * BN);
        issued = it + 1;
      }
      // Drain: every issued copy must have landed before the CTA may exit.
      for (int it = max(0, issued - C::STAGES); it < issued; ++it)
        mbar_wait(&full[it % C::STAGES], (it / C::STAGES) & 1, ea.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = EB == 2 ? make_idesc(BM, BN)
                                         : (DEQ ? make_idesc_f16(BM, BN) : make_idesc_e4m3(BM, BN));
      for (int it = 0; it < nk; ++it) {
        const int s = it % C::STAGES;
        const uint32_t ph = (it / C::STAGES) & 1;
        if (!mbar_wait(&full[s], ph, ea.status)) break;
        if (DEQ && !mbar_wait(&conv[it & 1], (it >> 1) & 1, ea.status)) break;
        tc_fence_after();
        const uint32_t sb = smem_u32(stages + s * C::STAGE);
        const uint32_t sa = DEQ ? smem_u32(aring + (it & 1) * C::A_BYTES) : sb;
        const uint64_t da = make_sdesc(sa), db = make_sdesc(sb + C::B_OFF);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          if (EB != 1)
            umma_bf16(tmem, da + 2 * kk, db + 2 * kk, idesc, (it > 0 || kk > 0) ? 1u : 0u);
          else
            umma_e4m3(tmem, da + 2 * kk, db + 2 * kk, idesc, (it > 0 || kk > 0) ? 1u : 0u);
        umma_commit(&empty[s]);
        if (DEQ) umma_commit(&afree[it & 1]);
      }
      umma_commit(tfull);
    }
  } else {
    if (DEQ) {
      // ------------------------- widen A to FP16 ---------------------------
      // 128 threads, four passes over the 8 KB E4M3 tile: thread t reads the
      // 16-byte piece i = 128 p + t (row i / 4, K elements 16 (i % 4) ..),
      // contiguous across the warp, and writes its two FP16 pieces into the
      // 128-byte-swizzled row (16-byte chunk c at c ^ (row % 8)).  (One
      // 8-byte read and one whole chunk per thread measured 15% slower.)
      const int ct = threadIdx.x - 64;
      for (int it = 0; it < nk; ++it) {
        const int s = it % C::STAGES;
        const uint32_t ph = (it / C::STAGES) & 1;
        if (!mbar_wait(&full[s], ph, ea.status)) break;
        // the A slot is free once the MMAs of K block it - 2 are done
        if (!mbar_wait(&afree[it & 1], ((it >> 1) & 1) ^ 1, ea.status)) break;
        uint8_t *sa = aring + (it & 1) * C::A_BYTES;
        const uint8_t *raw = stages + s * C::STAGE + C::RAW_OFF;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int i = 128 * p + ct;
          const int r = i >> 2, c2 = 2 * (i & 3);
          const uint4 in = *reinterpret_cast<const uint4 *>(raw + 16 * i);
          const uint32_t w[4] = {in.x, in.y, in.z, in.w};
          uint32_t o[8];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            o[2 * q] = cvt_e4m3x2_f16x2(w[q] & 0xFFFFu);
            o[2 * q + 1] = cvt_e4m3x2_f16x2(w[q] >> 16);
          }
          *reinterpret_cast<uint4 *>(sa + r * 128 + ((c2 ^ (r & 7)) << 4)) =
              make_uint4(o[0], o[1], o[2], o[3]);
          *reinterpret_cast<uint4 *>(sa + r * 128 + (((c2 + 1) ^ (r & 7)) << 4)) =
              make_uint4(o[4], o[5], o[6], o[7]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[it & 1]);
      }
    }
    // ------------------------------ epilogue ------------------------------
    const bool ok = mbar_wait(tfull, 0, ea.status);
    tc_fence_after();
    const int qd = warp & 3;
    const int row = m_tile * BM + qd * 32 + lane;
    const int ncol0 = n_tile * BN;
    double d2 = 0.0, cdr = 0.0;
    float d2f = 0.f, cdf = 0.f;
    if (EPI != E_SPLITK && EPI != E_SPLITB && EPI != E_VACC && EPI != E_F64 && row < M) {
      d2 = ea.Delta2[row];
      cdr = ea.cd[row];
    }
    if (EPI == E_SPLITB && row < M) {
      d2f = ea.d2f[row];
      cdf = ea.cdf[row];
    }
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0, r);
      if (!ok || nk == 0) {
#pragma unroll
        for (int i = 0; i < 32; ++i) r[i] = 0u;
      }
      if (EPI == E_SPLITK) {
        float *out = ea.ypart + (size_t)split * Ncols * ea.ldo;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int col = ncol0 + c0 + i;
          if (col < Ncols && row < M) out[(size_t)col * ea.ldo + row] = __uint_as_float(r[i]);
        }
      } else if (EPI == E_F64) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int col = ncol0 + c0 + i;
          if (col < Ncols && row < M) {
            double *o = ea.out + (size_t)col * ea.ldo + row;
            *o = (ea.add ? *o : 0.0) + (double)__uint_as_float(r[i]);
          }
        }
      } else if (EPI == E_VACC) {
        // FP32 accumulation of split-BF16 partial products (ea.ldo != 0: add)
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int col = ncol0 + c0 + i;
          if (col < Ncols && row < M) {
            float *o = ea.ucd + kblk_f32(col, row, Ncols);
            *o = (ea.ldo ? *o : 0.0f) + __uint_as_float(r[i]);
          }
        }
      } else if (EPI == E_SPLITB) {
        // c_K Delta^1/2 (L y), FP32, store only (the FP64 assembly of w and
        // the alpha estimate happen elsewhere; loads here would be scattered
        // 128-byte pieces across 256 vector rows)
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int col = ncol0 + c0 + i;
          if (col < Ncols && row < M) {
            const float cs = ea.colscale ? ea.colscale[col] : 1.0f;
            ea.ucd[kblk_f32(col, row, Ncols)] = cdf * (cs * __uint_as_float(r[i]));
          }
        }
      } else {
        double acc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int col = ncol0 + c0 + i;
          acc[i] = 0.0;
          if (col < Ncols && row < M) {
            const size_t o = (size_t)col * ea.N + row;
            const double u = (double)__uint_as_float(r[i]) *
                             (ea.colscale ? (double)ea.colscale[col] : 1.0);
            const double qv = ea.q[o];
            double wv = fma(d2, qv, cdr * u);
            if ((EPI == E_LANCZOS || EPI == E_LANCZOS_NA) && ea.qprev != nullptr)
              wv = fma(-ea.betaj[col], ea.qprev[o], wv);
            ea.w[o] = wv;
            acc[i] = qv * wv;
          }
        }
        if (EPI == E_LANCZOS) {
          warp_transpose_sum32(acc);
          red[qd * BN + c0 + lane] = acc[0];
        }
      }
    }
    if (EPI == E_LANCZOS) {
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const int te = threadIdx.x - 64;
      for (int col = te; col < BN; col += 128) {
        const int b = ncol0 + col;
        if (b < Ncols) {
          const double s = ((red[col] + red[BN + col]) + red[2 * BN + col]) + red[3 * BN + col];
          ea.alpha_part[(size_t)m_tile * Ncols + b] = s;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// Persistent form of the store-only contraction (ucd = c_K Delta^1/2 L y,
// the E_SPLITB epilogue): one CTA per SM walks the output tiles in launch
// order with the grid as stride.  Two TMEM accumulators (2 x BN columns)
// alternate, so the four epilogue warps drain tile i's accumulator while the
// MMA thread fills the other one with tile i + 1; the stage ring and its
// barrier phases run on across tiles, so TMA loads of the next tile start
// during the current tile's last MMAs.  Per output element the K order (the
// rotation by the M tile) is the one of k_gemm_tc, so results are
// bit-identical.  Every wait is bounded; on a timeout the loops stop, the
// producer still waits (bounded) for its own copies, and TMEM is freed.
template <int BN, int EB>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm_persist(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   int M, int Ncols, int num_kb, EpiArgs ea) {
  using C = Cfg<BN, 0>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::STAGES * C::STAGE);
  uint64_t *empty = full + C::STAGES;
  uint64_t *tfull = empty + C::STAGES;   // [2] accumulator a holds a finished tile
  uint64_t *tempty = tfull + 2;          // [2] the epilogue has drained accumulator a
  uint64_t *mdone = tempty + 2;          // every MMA issued by the CTA has completed
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mdone + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = (Ncols + BN - 1) / BN;
  const int m_tiles = (M + BM - 1) / BM;
  const int total = m_tiles * n_tiles;
  const int nk = num_kb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);   // one arrival per epilogue warp
    }
    mbar_init(mdone, 1);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tslot, 2 * C::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  auto tile_of = [&](int t, int &m_tile, int &n_tile) {
    if (ea.mfast) {
      m_tile = t % m_tiles;
      n_tile = t / m_tiles;
    } else {
      m_tile = t / n_tiles;
      n_tile = t % n_tiles;
    }
  };

  if (warp == 0) {
    if (lane == 0) {
      int it = 0, issued = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        int m_tile, n_tile;
        tile_of(t, m_tile, n_tile);
        for (int kk = 0; kk < nk; ++kk, ++it) {
          const int s = it % C::STAGES;
          const uint32_t ph = (it / C::STAGES) & 1;
          if (!mbar_wait(&empty[s], ph ^ 1, ea.status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], C::STAGE);
          uint8_t *sa = smem + s * C::STAGE;
          const int kb = (kk + (ea.rot ? m_tile : 0)) % nk;
          const int kx = kb * (BK * 2 / EB);
          tma_load_2d(sa, &tmA, &full[s], kx, m_tile * BM);
          tma_load_2d(sa + C::A_BYTES, &tmB, &full[s], kx, n_tile * BN);
          issued = it + 1;
        }
      }
      // every issued copy must have landed before the CTA may exit
      for (int i = max(0, issued - C::STAGES); i < issued; ++i)
        mbar_wait(&full[i % C::STAGES], (i / C::STAGES) & 1, ea.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = EB == 2 ? make_idesc(BM, BN) : make_idesc_e4m3(BM, BN);
      int it = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++i) {
        const int a = i & 1, use = i >> 1;
        if (use > 0 && !mbar_wait(&tempty[a], (use - 1) & 1, ea.status)) break;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(a * BN);
        for (int kk = 0; kk < nk; ++kk, ++it) {
          const int s = it % C::STAGES;
          const uint32_t ph = (it / C::STAGES) & 1;
          if (!mbar_wait(&full[s], ph, ea.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * C::STAGE);
          const uint64_t da = make_sdesc(sa), db = make_sdesc(sa + C::A_BYTES);
#pragma unroll
          for (int q = 0; q < BK / 16; ++q)
            if (EB == 2)
              umma_bf16(acc, da + 2 * q, db + 2 * q, idesc, (kk > 0 || q > 0) ? 1u : 0u);
            else
              umma_e4m3(acc, da + 2 * q, db + 2 * q, idesc, (kk > 0 || q > 0) ? 1u : 0u);
          umma_commit(&empty[s]);
        }
        if (ok) umma_commit(&tfull[a]);
      }
      // no MMA may still write TMEM when it is freed (also after a timeout)
      umma_commit(mdone);
      mbar_wait(mdone, 0, ea.status);
    }
  } else {
    // ------------------------------ epilogue ------------------------------
    const int qd = warp & 3;
    int i = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++i) {
      const int a = i & 1, use = i >> 1;
      if (!mbar_wait(&tfull[a], use & 1, ea.status)) break;
      tc_fence_after();
      int m_tile, n_tile;
      tile_of(t, m_tile, n_tile);
      const int row = m_tile * BM + qd * 32 + lane;
      const int ncol0 = n_tile * BN;
      const float cdf = row < M ? ea.cdf[row] : 0.f;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (uint32_t)(a * BN) + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0, r);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int col = ncol0 + c0 + q;
          if (col < Ncols && row < M) {
            const float cs = ea.colscale ? ea.colscale[col] : 1.0f;
            ea.ucd[kblk_f32(col, row, Ncols)] = cdf * (cs * __uint_as_float(r[q]));
          }
        }
      }
      // the accumulator may be refilled once all four warps have read it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[a]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * C::TMEM_COLS);
  }
}

// Yh = bf16(sum_p Ypart[p]) in fixed order; optionally per-block partials of
// sum_mu y_mu Yh_mu (grid: A/256 blocks per vector row).
__global__ void k_reduce_y_bf16(const float *__restrict__ Ypart, int splits, int Bs, int A,
                                __nv_bfloat16 *__restrict__ Yh, float *__restrict__ yy,
                                const double *__restrict__ vscale) {
  __shared__ float red[8];
  const int b = blockIdx.y;
  const int mu = blockIdx.x * 256 + threadIdx.x;
  const size_t n = (size_t)Bs * A;
  float s = 0.0f;
  const size_t i = (size_t)b * A + mu;
  if (mu < A) {
    for (int p = 0; p < splits; ++p) s += Ypart[(size_t)p * n + i];
    // a contraction of an unnormalised vector: scale to the normalised one
    if (vscale != nullptr) s *= (float)vscale[b];
    const __nv_bfloat16 hq = __float2bfloat16_rn(s);
    Yh[i] = hq;
    s *= __bfloat162float(hq);
  } else {
    s = 0.0f;
  }
  if (yy != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
      for (int w = 0; w < 8; ++w) t += red[w];
      yy[(size_t)b * gridDim.x + blockIdx.x] = t;
    }
  }
}

// Diagnostic of the bounded wait: thread 0 waits on a fresh barrier with
// the given limit; with `arrive`, thread 1 completes the barrier's phase
// first, otherwise nothing does and the wait must run out and set
// ST_TIMEOUT.  No asynchronous copy references the barrier.
__global__ void k_wait_selftest(int arrive, long long limit, unsigned *status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 1) mbar_arrive(&bar);
  if (threadIdx.x == 0) mbar_wait_for(&bar, 0, status, limit);
  __syncthreads();
  if (threadIdx.x == 0) mbar_inval(&bar);
}

}  // namespace tc

void launch_wait_selftest(int arrive, long long limit_cycles, unsigned *status, cudaStream_t st) {
  tc::k_wait_selftest<<<1, 32, 0, st>>>(arrive, limit_cycles, status);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct TcPlan {
  CUtensorMap g1A, g1B, g2A, g2B, g2Alo;
  // E4M3 operands (fp8 plans): L8t / x8 for gemm1, L8 / y8 for gemm2
  CUtensorMap f1A, f1B, f2A, f2B;
  // E4M3 L widened to FP16 in shared memory (deq plans): raw L8t / x16 for
  // gemm1, raw L8 / y16 for gemm2
  CUtensorMap d1A, d1B, d2A, d2B;
  bool fp8 = false;
  bool deq = false;
  const uint16_t *x16 = nullptr, *y16 = nullptr;
  bool has_bf16 = false;   // g1A / g2A / g2Alo encoded (the system has BF16 copies)
  const uint8_t *x8 = nullptr, *y8 = nullptr;
  const float *ty = nullptr;   // per-vector scale of y8 (gemm2 column scale)
  int BN1, BN2;   // N tile of gemm1 / gemm2 (and the coupling products)
  int rot1 = 1;   // gemm1 K-start rotation (tuned); gemm2 always rotates
  int mfast2 = 0; // gemm2 tile numbering (EpiArgs::mfast), tuned
  int half2 = 0;  // gemm2 pipeline, tuned: 0 one CTA per tile, 1 half depth (two CTAs
                  // per SM), 2 persistent with two TMEM accumulators
  const __nv_bfloat16 *xh;
  int N, A, Bs;
  int splits, kb_per_split;
  float *ypart;
  __nv_bfloat16 *yh;
  const double *Delta2, *cd;
  const float *d2f, *cdf;
};

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  std::call_once(g_encode_once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return g_encode;
}

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && get_encode() != nullptr;
}

// 2-D K-major tensor map: inner (K) extent, outer rows, a box of one
// 128-byte swizzle row (64 BF16 or 128 E4M3 elements) by box_outer rows.
// elem_bytes 3: FP16 elements (2 bytes).
static CUtensorMapDataType map_dtype(int elem_bytes) {
  return elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                         : (elem_bytes == 3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                            : CU_TENSOR_MAP_DATA_TYPE_UINT8);
}
static int map_bytes(int elem_bytes) { return elem_bytes == 1 ? 1 : 2; }

static bool encode_2d(CUtensorMap *tm, const void *base, uint64_t inner, uint64_t outer,
                      uint32_t box_outer, uint64_t row_elems = 0, int elem_bytes = 2) {
  auto enc = get_encode();
  if (!enc) return false;
  const int eb = map_bytes(elem_bytes);
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {(row_elems ? row_elems : inner) * (uint64_t)eb};
  cuuint32_t box[2] = {(cuuint32_t)(128 / eb), box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(tm, map_dtype(elem_bytes), 2, const_cast<void *>(base), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// E4M3 A operand of the widening kernels: a box of 64 bytes by BM rows, not
// swizzled (row r of the box at r * 64 in shared memory).  kblk: the
// K-block-major layout (kblk_e4m3; the box is half of a 128-byte K-block
// row, x = 0 or 64); else row-major [outer][inner].
static bool encode_raw_a(CUtensorMap *tm, const uint8_t *base, uint64_t inner, uint64_t outer,
                         bool kblk) {
  auto enc = get_encode();
  if (!enc) return false;
  CUresult r;
  if (kblk) {
    cuuint64_t dims[3] = {128, outer, inner / 128};
    cuuint64_t strides[2] = {128, outer * 128};
    cuuint32_t box[3] = {64, (cuuint32_t)tc::BM, 1};
    cuuint32_t es[3] = {1, 1, 1};
    r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(base), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner};
    cuuint32_t box[2] = {64, (cuuint32_t)tc::BM};
    cuuint32_t es[2] = {1, 1};
    r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(base), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return r == CUDA_SUCCESS;
}

// 3-D map of a K-block-major operand (kblk_bf16 / kblk_e4m3): dims (one
// 128-byte row of elements, rows, K blocks), box (128 bytes, box_rows, 1);
// each box is one contiguous 128 x box_rows-byte run, swizzled into the
// same shared-memory image as the 2-D row-major box.
static bool encode_kblk(CUtensorMap *tm, const void *base, uint64_t kblocks, uint64_t rows,
                        uint32_t box_rows, int elem_bytes = 2) {
  auto enc = get_encode();
  if (!enc) return false;
  const int eb = map_bytes(elem_bytes);
  cuuint64_t dims[3] = {(cuuint64_t)(128 / eb), rows, kblocks};
  cuuint64_t strides[2] = {128, rows * 128};
  cuuint32_t box[3] = {(cuuint32_t)(128 / eb), box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(tm, map_dtype(elem_bytes), 3, const_cast<void *>(base), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int choose_splits(int tiles, int num_kb, int nsm) {
  // Fill whole waves of one CTA per SM: pick the split count whose CTA total
  // wastes the least of its last wave, with at least 8 K blocks per split.
  int best = 1;
  double best_cost = 1e30;
  for (int s = 1; s <= 64; ++s) {
    int per = (num_kb + s - 1) / s;
    if (per < 8 && s > 1) break;
    int real_s = (num_kb + per - 1) / per;
    int ctas = tiles * real_s;
    int waves = (ctas + nsm - 1) / nsm;
    double cost = (double)waves * per;   // time ~ waves x K blocks per CTA
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = real_s;
    }
  }
  return best;
}

int tc_n_mt(const SysDev &s) { return s.N / tc::BM; }

TcPlan *tc_plan_create(const SysDev &s, int Bs, const __nv_bfloat16 *xh, float *ypart,
                       __nv_bfloat16 *yh, int *splits_out, char *err, size_t errn) {
  TcPlan *p = new TcPlan();
  p->N = s.N;
  p->A = s.A;
  p->Bs = Bs;
  p->BN1 = p->BN2 = Bs >= 256 ? 256 : (Bs >= 128 ? 128 : 64);
  p->xh = xh;
  if (Bs < 64 || s.A < tc::BM || s.N < tc::BM) {
    snprintf(err, errn, "tensor-core plan needs Bs >= 64, N_aux and N_vc padded >= 128");
    delete p;
    return nullptr;
  }
  int nsm = 148;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int num_kb = s.N / tc::BK;
  const int tiles1 = ((s.A + tc::BM - 1) / tc::BM) * ((Bs + p->BN1 - 1) / p->BN1);
  p->splits = choose_splits(tiles1, num_kb, nsm);
  p->kb_per_split = (num_kb + p->splits - 1) / p->splits;
  p->splits = (num_kb + p->kb_per_split - 1) / p->kb_per_split;
  p->ypart = ypart;
  p->yh = yh;
  p->Delta2 = s.Delta2;
  p->cd = s.cd;
  p->d2f = s.d2f;
  p->cdf = s.cdf;
  // the BF16 copies of L are absent for a system prepared without them
  // (E4M3 plans); their maps stay unset then
  bool ok = encode_kblk(&p->g1B, xh, (uint64_t)s.N / 64, (uint64_t)Bs, (uint32_t)p->BN1) &&
            encode_2d(&p->g2B, yh, (uint64_t)s.A, (uint64_t)Bs, (uint32_t)p->BN2);
  if (ok && s.Lb) {
    ok = encode_kblk(&p->g1A, s.Ltb, (uint64_t)s.N / 64, (uint64_t)s.A, tc::BM) &&
         encode_2d(&p->g2A, s.Lb, (uint64_t)s.A, (uint64_t)s.N, tc::BM) &&
         encode_2d(&p->g2Alo, s.Lb_lo, (uint64_t)s.A, (uint64_t)s.N, tc::BM);
    p->has_bf16 = ok;
  }
  if (!ok) {
    snprintf(err, errn, "cuTensorMapEncodeTiled failed");
    delete p;
    return nullptr;
  }
  if (splits_out) *splits_out = p->splits;
  return p;
}

void tc_plan_destroy(TcPlan *p) { delete p; }

template <int BN, int EPI, int EB = 2, int HALF = 0>
static void launch_tc(const CUtensorMap &A, const CUtensorMap &B, int M, int Ncols, int num_kb,
                      int kb_per_split, int splits, const tc::EpiArgs &ea, cudaStream_t st) {
  using C = tc::Cfg<BN, HALF, EB == 3>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(tc::k_gemm_tc<BN, EPI, EB, HALF>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    attr_done = true;
  }
  dim3 grid((M + tc::BM - 1) / tc::BM, (Ncols + BN - 1) / BN, splits);
  tc::k_gemm_tc<BN, EPI, EB, HALF><<<grid, tc::NTHREADS, C::SMEM, st>>>(A, B, M, Ncols, num_kb,
                                                                        kb_per_split, ea);
}

template <int BN, int EB>
static void launch_persist(const CUtensorMap &A, const CUtensorMap &B, int M, int Ncols,
                           int num_kb, const tc::EpiArgs &ea, cudaStream_t st) {
  using C = tc::Cfg<BN, 0>;
  static bool attr_done = false;
  static int nsm = 0;
  if (!attr_done) {
    cudaFuncSetAttribute(tc::k_gemm_persist<BN, EB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         C::SMEM);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    attr_done = true;
  }
  const int total = ((M + tc::BM - 1) / tc::BM) * ((Ncols + BN - 1) / BN);
  const int grid = std::max(1, std::min(total, nsm > 0 ? nsm : 148));
  tc::k_gemm_persist<BN, EB><<<grid, tc::NTHREADS, C::SMEM, st>>>(A, B, M, Ncols, num_kb, ea);
}

// half: 1 = the half-depth pipeline (two CTAs per SM), 2 = the persistent
// kernel with two accumulators; store-only epilogue only, and not for the
// widening kernels (their epilogue warps convert during the main loop)
template <int EPI, int EB = 2>
static void dispatch_bn(int BN, const CUtensorMap &A, const CUtensorMap &B, int M, int Ncols,
                        int num_kb, int kb_per_split, int splits, const tc::EpiArgs &ea,
                        cudaStream_t st, int half = 0) {
  if constexpr (EPI == tc::E_SPLITB && EB != 3) {
    if (half == 2 && splits == 1 && kb_per_split == num_kb) {
      if (BN == 256)
        launch_persist<256, EB>(A, B, M, Ncols, num_kb, ea, st);
      else if (BN == 128)
        launch_persist<128, EB>(A, B, M, Ncols, num_kb, ea, st);
      else
        launch_persist<64, EB>(A, B, M, Ncols, num_kb, ea, st);
      return;
    }
    if (half) {
      if (BN == 256)
        launch_tc<256, EPI, EB, 1>(A, B, M, Ncols, num_kb, kb_per_split, splits, ea, st);
      else if (BN == 128)
        launch_tc<128, EPI, EB, 1>(A, B, M, Ncols, num_kb, kb_per_split, splits, ea, st);
      else
        launch_tc<64, EPI, EB, 1>(A, B, M, Ncols, num_kb, kb_per_split, splits, ea, st);
      return;
    }
  }
  if (BN == 256)
    launch_tc<256, EPI, EB>(A, B, M, Ncols, num_kb, kb_per_split, splits, ea, st);
  else if (BN == 128)
    launch_tc<128, EPI, EB>(A, B, M, Ncols, num_kb, kb_per_split, splits, ea, st);
  else
    launch_tc<64, EPI, EB>(A, B, M, Ncols, num_kb, kb_per_split, splits, ea, st);
}

void launch_gemm1_tc(const TcPlan *p, unsigned *status, cudaStream_t st) {
  tc::EpiArgs ea{};
  ea.ypart = p->ypart;
  ea.ldo = p->A;
  ea.status = status;
  ea.rot = p->rot1;
  ea.a3 = ea.b3 = 1;   // L^T and X are K-block-major
  if (p->deq) {
    dispatch_bn<tc::E_SPLITK, 3>(p->BN1, p->d1A, p->d1B, p->A, p->Bs, p->N / tc::BK,
                                 p->kb_per_split, p->splits, ea, st);
    return;
  }
  if (p->fp8) {
    // same split count; K blocks of 128 elements
    const int nkb = p->N / 128;
    const int per = (nkb + p->splits - 1) / p->splits;
    dispatch_bn<tc::E_SPLITK, 1>(p->BN1, p->f1A, p->f1B, p->A, p->Bs, nkb, per, p->splits, ea,
                                 st);
    return;
  }
  if (!p->has_bf16) return;   // callers check tc_plan_has_bf16 first
  dispatch_bn<tc::E_SPLITK>(p->BN1, p->g1A, p->g1B, p->A, p->Bs, p->N / tc::BK, p->kb_per_split,
                            p->splits, ea, st);
}

void launch_reduce_y_bf16(const float *Ypart, int splits, int Bs, int A, __nv_bfloat16 *Yh,
                          float *yy, cudaStream_t st, const double *vscale) {
  dim3 grid((A + 255) / 256, Bs);
  tc::k_reduce_y_bf16<<<grid, 256, 0, st>>>(Ypart, splits, Bs, A, Yh, yy, vscale);
}

void launch_gemm2_tc(const TcPlan *p, int epi, const double *q, const double *qprev,
                     const double *betaj, double *w, double *alpha_part, unsigned *status,
                     cudaStream_t st) {
  tc::EpiArgs ea{};
  ea.rot = 1;
  ea.N = p->N;
  ea.Delta2 = p->Delta2;
  ea.cd = p->cd;
  ea.q = q;
  ea.qprev = qprev;
  ea.betaj = betaj;
  ea.w = w;
  ea.alpha_part = alpha_part;
  ea.status = status;
  if (p->deq) {
    ea.colscale = p->ty;
    const int nkb = p->A / tc::BK;
    if (epi == EPI_LANCZOS && alpha_part == nullptr)
      dispatch_bn<tc::E_LANCZOS_NA, 3>(p->BN2, p->d2A, p->d2B, p->N, p->Bs, nkb, nkb, 1, ea, st);
    else if (epi == EPI_LANCZOS)
      dispatch_bn<tc::E_LANCZOS, 3>(p->BN2, p->d2A, p->d2B, p->N, p->Bs, nkb, nkb, 1, ea, st);
    else
      dispatch_bn<tc::E_APPLY, 3>(p->BN2, p->d2A, p->d2B, p->N, p->Bs, nkb, nkb, 1, ea, st);
    return;
  }
  if (p->fp8) {
    ea.colscale = p->ty;
    const int nkb = p->A / 128;
    if (epi == EPI_LANCZOS && alpha_part == nullptr)
      dispatch_bn<tc::E_LANCZOS_NA, 1>(p->BN2, p->f2A, p->f2B, p->N, p->Bs, nkb, nkb, 1, ea, st);
    else if (epi == EPI_LANCZOS)
      dispatch_bn<tc::E_LANCZOS, 1>(p->BN2, p->f2A, p->f2B, p->N, p->Bs, nkb, nkb, 1, ea, st);
    else
      dispatch_bn<tc::E_APPLY, 1>(p->BN2, p->f2A, p->f2B, p->N, p->Bs, nkb, nkb, 1, ea, st);
    return;
  }
  if (!p->has_bf16) return;
  const int num_kb = p->A / tc::BK;
  if (epi == EPI_LANCZOS && alpha_part == nullptr)
    dispatch_bn<tc::E_LANCZOS_NA>(p->BN2, p->g2A, p->g2B, p->N, p->Bs, num_kb, num_kb, 1, ea, st);
  else if (epi == EPI_LANCZOS)
    dispatch_bn<tc::E_LANCZOS>(p->BN2, p->g2A, p->g2B, p->N, p->Bs, num_kb, num_kb, 1, ea, st);
  else
    dispatch_bn<tc::E_APPLY>(p->BN2, p->g2A, p->g2B, p->N, p->Bs, num_kb, num_kb, 1, ea, st);
}

namespace tc {
// bf16 hi / lo halves of M rows into a zero-padded [Bs][A] operand.
__global__ void k_split_m(const double *__restrict__ M, int nvec, int n_aux, int Bs, int A,
                          int lo, __nv_bfloat16 *__restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)Bs * A) return;
  const int b = (int)(i / A), mu = (int)(i - (size_t)b * A);
  float v = 0.0f;
  if (b < nvec && mu < n_aux) {
    const double x = M[(size_t)b * n_aux + mu];
    const __nv_bfloat16 hi = __double2bfloat16(x);
    v = lo ? (float)(x - (double)__bfloat162float(hi)) : __bfloat162float(hi);
  }
  out[i] = __float2bfloat16_rn(v);
}
}  // namespace tc

bool launch_coupling_tc(const TcPlan *p, const SysDev &s, const double *M, int nvec,
                        float *vf, unsigned *status, cudaStream_t st) {
  if (!p->has_bf16) return false;
  const size_t n = (size_t)p->Bs * p->A;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  tc::EpiArgs ea{};
  ea.rot = 1;
  ea.N = p->N;
  ea.ucd = vf;
  ea.status = status;
  const int num_kb = p->A / tc::BK;
  // L_hi M_hi, then + L_hi M_lo, then + L_lo M_hi
  tc::k_split_m<<<blocks, 256, 0, st>>>(M, nvec, s.n_aux, p->Bs, p->A, 0, p->yh);
  ea.ldo = 0;
  dispatch_bn<tc::E_VACC>(p->BN2, p->g2A, p->g2B, p->N, p->Bs, num_kb, num_kb, 1, ea, st);
  ea.ldo = 1;
  dispatch_bn<tc::E_VACC>(p->BN2, p->g2Alo, p->g2B, p->N, p->Bs, num_kb, num_kb, 1, ea, st);
  tc::k_split_m<<<blocks, 256, 0, st>>>(M, nvec, s.n_aux, p->Bs, p->A, 1, p->yh);
  dispatch_bn<tc::E_VACC>(p->BN2, p->g2A, p->g2B, p->N, p->Bs, num_kb, num_kb, 1, ea, st);
  return true;
}

void launch_gemm2_tc_split(const TcPlan *p, float *ucd, unsigned *status, cudaStream_t st) {
  tc::EpiArgs ea{};
  ea.rot = 1;
  ea.mfast = p->mfast2;
  ea.N = p->N;
  ea.cdf = p->cdf;
  ea.ucd = ucd;
  ea.status = status;
  if (p->deq) {
    ea.colscale = p->ty;
    const int nkb = p->A / tc::BK;
    dispatch_bn<tc::E_SPLITB, 3>(p->BN2, p->d2A, p->d2B, p->N, p->Bs, nkb, nkb, 1, ea, st);
    return;
  }
  if (p->fp8) {
    ea.colscale = p->ty;
    const int nkb = p->A / 128;
    dispatch_bn<tc::E_SPLITB, 1>(p->BN2, p->f2A, p->f2B, p->N, p->Bs, nkb, nkb, 1, ea, st,
                                 p->half2);
    return;
  }
  if (!p->has_bf16) return;
  const int num_kb = p->A / tc::BK;
  dispatch_bn<tc::E_SPLITB>(p->BN2, p->g2A, p->g2B, p->N, p->Bs, num_kb, num_kb, 1, ea, st,
                            p->half2);
}

// out (=, or += if add) sum_{p < np} A_p B_p^T with A_p [M][K], B_p [Ncols][K]
// BF16 row-major (K contiguous), or A_p K-block-major (kblk_bf16 over M
// rows) where a_kblk[p] != 0; FP32 accumulation in tensor memory over K
// chunks of at most kchunk, each chunk added to the FP64 output.
// out[col * ldo + row].  K % 8 == 0 (16-byte TMA row stride); K % 64 == 0
// for a K-block-major operand.
bool tc_gemm_f64out(int np, const __nv_bfloat16 *const *A, const int *a_kblk,
                    const __nv_bfloat16 *const *B, int M, int Ncols, int K, int kchunk,
                    double *out, int ldo, int add, unsigned *status, cudaStream_t st, char *err,
                    size_t errn) {
  bool any_kblk = false;
  for (int p = 0; p < np; ++p) any_kblk = any_kblk || (a_kblk && a_kblk[p]);
  if (K % 8 != 0 || kchunk % tc::BK != 0 || kchunk <= 0 || (any_kblk && K % tc::BK != 0)) {
    snprintf(err, errn, "tc_gemm_f64out: K = %d not a multiple of 8 (64 K-block-major) or bad chunk", K);
    return false;
  }
  tc::EpiArgs ea{};
  ea.rot = 1;
  ea.out = out;
  ea.ldo = ldo;
  ea.status = status;
  bool first = add == 0;
  for (int k0 = 0; k0 < K; k0 += kchunk) {
    const int kc = std::min(kchunk, K - k0);
    for (int p = 0; p < np; ++p) {
      CUtensorMap ta, tb;
      const bool kb = a_kblk && a_kblk[p];
      const bool ta_ok =
          kb ? encode_kblk(&ta, A[p] + (size_t)(k0 / tc::BK) * M * tc::BK, (uint64_t)kc / tc::BK,
                           (uint64_t)M, tc::BM)
             : encode_2d(&ta, A[p] + k0, (uint64_t)kc, (uint64_t)M, tc::BM, (uint64_t)K);
      ea.a3 = kb ? 1 : 0;
      if (!ta_ok || !encode_2d(&tb, B[p] + k0, (uint64_t)kc, (uint64_t)Ncols, 256, (uint64_t)K)) {
        snprintf(err, errn, "cuTensorMapEncodeTiled failed (tc_gemm_f64out)");
        return false;
      }
      ea.add = first ? 0 : 1;
      first = false;
      const int nkb = (kc + tc::BK - 1) / tc::BK;
      launch_tc<256, tc::E_F64>(ta, tb, M, Ncols, nkb, nkb, 1, ea, st);
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Autotuner: the N tile of each contraction and the split count of gemm1 are
// timed on the plan's own operands (CUDA events, best of 3 after a warm-up)
// and cached per (device, N, A, Bs).  A candidate replaces the heuristic
// choice only when it is more than 3% faster.  LGW_AUTOTUNE=0 disables it.
// ---------------------------------------------------------------------------
namespace {
struct TuneKey {
  int dev, N, A, Bs, fp8;
  bool operator<(const TuneKey &o) const {
    if (fp8 != o.fp8) return fp8 < o.fp8;
    if (dev != o.dev) return dev < o.dev;
    if (N != o.N) return N < o.N;
    if (A != o.A) return A < o.A;
    return Bs < o.Bs;
  }
};
struct TuneVal {
  int BN1, splits, BN2, rot1, mfast2, half2;
};
std::map<TuneKey, TuneVal> g_tune;
std::mutex g_tune_mu;

bool plan_encode_b(TcPlan *p) {
  bool ok = encode_kblk(&p->g1B, p->xh, (uint64_t)p->N / 64, (uint64_t)p->Bs, (uint32_t)p->BN1) &&
            encode_2d(&p->g2B, p->yh, (uint64_t)p->A, (uint64_t)p->Bs, (uint32_t)p->BN2);
  if (ok && p->fp8)
    ok = encode_kblk(&p->f1B, p->x8, (uint64_t)p->N / 128, (uint64_t)p->Bs, (uint32_t)p->BN1, 1) &&
         encode_2d(&p->f2B, p->y8, (uint64_t)p->A, (uint64_t)p->Bs, (uint32_t)p->BN2, 0, 1);
  if (ok && p->deq)
    ok = encode_kblk(&p->d1B, p->x16, (uint64_t)p->N / 64, (uint64_t)p->Bs, (uint32_t)p->BN1, 3) &&
         encode_2d(&p->d2B, p->y16, (uint64_t)p->A, (uint64_t)p->Bs, (uint32_t)p->BN2, 0, 3);
  return ok;
}

void plan_set_splits(TcPlan *p, int splits) {
  const int num_kb = p->N / tc::BK;
  p->kb_per_split = (num_kb + splits - 1) / splits;
  p->splits = (num_kb + p->kb_per_split - 1) / p->kb_per_split;
}

template <class F>
float time_best(F &&f, cudaStream_t st) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  f();   // warm-up
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(a, st);
    f();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}
}  // namespace

// LGW_GEMM2_PIPE = 0, 1 or 2 forces GEMM2's pipeline variant (one CTA per
// tile, half depth, persistent) after tuning; every variant gives the same
// bits, so this only serves tests and measurements.
static void apply_gemm2_override(TcPlan *p) {
  const char *e = getenv("LGW_GEMM2_PIPE");
  if (e && e[0] >= '0' && e[0] <= '2' && e[1] == '\0') p->half2 = e[0] - '0';
}

bool tc_plan_autotune(TcPlan *p, float *ucd, unsigned *status, cudaStream_t st, int *splits_out) {
  const char *env = getenv("LGW_AUTOTUNE");
  if (env && env[0] == '0') {
    apply_gemm2_override(p);
    return true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  const TuneKey key{dev, p->N, p->A, p->Bs, p->deq ? 2 : (p->fp8 ? 1 : 0)};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      p->BN1 = it->second.BN1;
      p->BN2 = it->second.BN2;
      p->rot1 = it->second.rot1;
      p->mfast2 = it->second.mfast2;
      p->half2 = it->second.half2;
      apply_gemm2_override(p);
      plan_set_splits(p, it->second.splits);
      if (splits_out) *splits_out = p->splits;
      return plan_encode_b(p);
    }
  }
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int num_kb = p->N / tc::BK;
  const int bn_max = p->Bs >= 256 ? 256 : (p->Bs >= 128 ? 128 : 64);
  auto gemm1 = [&]() {
    launch_gemm1_tc(p, status, st);
    launch_reduce_y_bf16(p->ypart, p->splits, p->Bs, p->A, p->yh, nullptr, st);
  };
  // gemm1: N tile x split count x K-start rotation
  const TuneVal def{p->BN1, p->splits, p->BN2, p->rot1, p->mfast2, p->half2};
  float t_def = time_best(gemm1, st);
  TuneVal best = def;
  float t_best = t_def;
  for (int bn = 64; bn <= bn_max; bn *= 2) {
    const int tiles = ((p->A + tc::BM - 1) / tc::BM) * ((p->Bs + bn - 1) / bn);
    const int s0 = choose_splits(tiles, num_kb, nsm);
    const int cands[3] = {std::max(1, s0 / 2), s0, std::min(64, 2 * s0)};
    for (int ci = 0; ci < 3; ++ci)
      for (int rot = 0; rot <= 1; ++rot) {
        const int sreq = cands[ci];
        if (num_kb / sreq < 8 && sreq > 1) continue;
        p->BN1 = bn;
        p->rot1 = rot;
        plan_set_splits(p, sreq);
        if (bn == def.BN1 && p->splits == def.splits && rot == def.rot1) continue;
        if (!plan_encode_b(p)) return false;
        const float t = time_best(gemm1, st);
        if (t < t_best) {
          t_best = t;
          best.BN1 = bn;
          best.splits = p->splits;
          best.rot1 = rot;
        }
      }
  }
  if (t_best > 0.97f * t_def) {
    best.BN1 = def.BN1;
    best.splits = def.splits;
    best.rot1 = def.rot1;
  }
  p->BN1 = best.BN1;
  p->rot1 = best.rot1;
  plan_set_splits(p, best.splits);
  // gemm2 (store-only epilogue into the caller's scratch): N tile x tile
  // numbering x pipeline depth
  if (ucd != nullptr) {
    auto gemm2 = [&]() { launch_gemm2_tc_split(p, ucd, status, st); };
    if (!plan_encode_b(p)) return false;
    const float t2_def = time_best(gemm2, st);
    float t2_best = t2_def;
    for (int bn = 64; bn <= bn_max; bn *= 2)
      for (int mf = 0; mf <= 1; ++mf)
        for (int hf = 0; hf <= (p->deq ? 0 : 2); ++hf) {
          if (bn == def.BN2 && mf == def.mfast2 && hf == def.half2) continue;
          p->BN2 = bn;
          p->mfast2 = mf;
          p->half2 = hf;
          if (!plan_encode_b(p)) return false;
          const float t = time_best(gemm2, st);
          if (t < t2_best) {
            t2_best = t;
            best.BN2 = bn;
            best.mfast2 = mf;
            best.half2 = hf;
          }
        }
    if (t2_best > 0.97f * t2_def) {
      best.BN2 = def.BN2;
      best.mfast2 = def.mfast2;
      best.half2 = def.half2;
    }
    p->BN2 = best.BN2;
    p->mfast2 = best.mfast2;
    p->half2 = best.half2;
  }
  if (!plan_encode_b(p)) return false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  apply_gemm2_override(p);
  if (splits_out) *splits_out = p->splits;
  return cudaGetLastError() == cudaSuccess;
}

// Switch a plan to E4M3 operands: L8t [A][N] and x8 [Bs][N] (K-block-major) for gemm1, L8
// [N][A] and y8 [Bs][A] for gemm2 (ty: per-vector scale of y8).
bool tc_plan_enable_fp8(TcPlan *p, const uint8_t *L8t, const uint8_t *L8, const uint8_t *x8,
                        const uint8_t *y8, const float *ty) {
  p->fp8 = true;
  p->x8 = x8;
  p->y8 = y8;
  p->ty = ty;
  return encode_kblk(&p->f1A, L8t, (uint64_t)p->N / 128, (uint64_t)p->A, tc::BM, 1) &&
         encode_2d(&p->f2A, L8, (uint64_t)p->A, (uint64_t)p->N, tc::BM, 0, 1) &&
         plan_encode_b(p);
}

// Switch a plan to E4M3 L widened to FP16 in shared memory: raw L8t [A][N]
// (K-block-major) with x16 [Bs][N] (FP16, K-block-major like xh) for gemm1,
// raw L8 [N][A] with y16 [Bs][A] (FP16) for gemm2 (ty: per-vector scale of
// y16).
bool tc_plan_enable_deq(TcPlan *p, const uint8_t *L8t, const uint8_t *L8, const uint16_t *x16,
                        const uint16_t *y16, const float *ty) {
  p->deq = true;
  p->half2 = 0;
  p->x16 = x16;
  p->y16 = y16;
  p->ty = ty;
  return encode_raw_a(&p->d1A, L8t, (uint64_t)p->N, (uint64_t)p->A, true) &&
         encode_raw_a(&p->d2A, L8, (uint64_t)p->A, (uint64_t)p->N, false) && plan_encode_b(p);
}

bool tc_plan_has_bf16(const TcPlan *p) { return p->has_bf16; }

}  // namespace lgw
