// Tensor-core sketch with FP64 accuracy (Algorithm 1/2 step 3 on tcgen05).
//
// C = Gamma^T X (C: S x Q FP64, Gamma: L x S, X: L x Q FP64 row-major) is
// computed from exact bf16 "digit" slices of both operands:
//   Gamma = 2^-12 q, q integer, |q| <= 32767:  q = 256 h + g_lo,  |h|, |g_lo| <= 128
//   X[l, j] = 2^(e_j - 7) sum_{p=1..8} d_p[l, j] 2^(-8(p-1))  (+ |residual| <= 2^(e_j - 64))
// with e_j a per-column (per-segment) exponent, |d_p| <= 128.  All digits are
// integers of at most 8 bits, exact in bf16, so every tcgen05.mma product is
// exact and an FP32 sum of up to 512 rows of two such products stays below
// 2^24 and is exact too.  Products of equal weight form eight groups
//   g = 0:  h d_1;   g >= 1:  h d_{g+1} + g_lo d_g,     weight 2^(e_j - 11 - 8 g)
// (g_lo d_8, at most 2^(e_j - 61) per row, is dropped).  Each group is accumulated
// exactly in TMEM over a chunk of 512 rows; the chunk's group sums (integers
// below 2^24) are added exactly into two int64 accumulators per column, so
// the only rounding of the whole segment is the final conversion to FP64,
// while the multiplications run on the tensor cores.
//
// Operands are split into digit planes in global memory one segment of rows at
// a time (K-major, bf16; the digits of X are cut from its 64-bit fixed-point
// form with integer shifts), then a 128 x 64 output tile per CTA streams them
// through a two-stage shared-memory ring into tcgen05.mma (M=128, K=16, FP32
// accumulators in TMEM, 8 groups x 64 columns; four MMAs per K-step, N = 256,
// 256, 256 and 192, each spanning the consecutive groups of four digit tiles).  The planes are stored as
// pre-swizzled tiles, so each stage is ten contiguous bulk copies
// (cp.async.bulk with mbarrier transaction counts).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

namespace {

constexpr int TC_M = 128;              // sketch rows per tile
constexpr int TC_N = 64;               // columns of X per tile
constexpr int TC_KT = 64;              // K per pipeline stage (one 128-byte swizzle row)
constexpr int TC_CHUNK = 512;          // rows summed exactly in TMEM before the int64 fold
constexpr int TC_GROUPS = 8;
constexpr int TC_DIGITS = 8;
constexpr int TC_THREADS = 256;              // two warpgroups share the TMEM lane quadrants
constexpr int TILE_A_BYTES = TC_M * TC_KT * 2;     // 16 KB
constexpr int TILE_B_BYTES = TC_N * TC_KT * 2;     // 8 KB
constexpr int STAGE_BYTES = 2 * TILE_A_BYTES + TC_DIGITS * TILE_B_BYTES;   // 96 KB
constexpr int TC_SMEM = 2 * STAGE_BYTES + 1024 + 64;
constexpr long long kSpinLimit = 1ll << 26;         // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait with an iteration limit; on timeout record the failure and return false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (long long it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}

// Wait bounded by elapsed time on the global timer (ns); on timeout record the
// failure and return false.
__device__ __forceinline__ bool mbar_wait_ns(uint64_t* bar, uint32_t parity, int* err,
                                             uint64_t limit_ns) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 63) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > limit_ns) break;
    }
  }
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                       // leading byte offset (unused with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset
  d |= (uint64_t)1 << 46;                       // descriptor version
  d |= (uint64_t)2 << 61;                       // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// Digit planes are stored as tiles: tile (row / R, k / 64) of a plane is a
// contiguous block of R x 64 bf16 (R = 128 for Gamma, 64 for X), laid out in
// 128-byte rows with the 16-byte chunks XOR-swizzled by (row % 8) -- the
// shared-memory layout the MMA descriptors read -- so one bulk copy moves a
// tile from HBM/L2 into a pipeline stage unchanged.
__host__ __device__ __forceinline__ int64_t tiled_off(int64_t row, int64_t k, int R, int64_t nkt) {
  const int64_t tile = (row / R) * nkt + (k >> 6);
  const int r = (int)(row % R), kk = (int)(k & 63);
  return tile * (int64_t)(R * 64) + (int64_t)r * 64 + ((((kk >> 3) ^ (r & 7))) << 3) + (kk & 7);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Per-column exponent of a segment: e_j with max_l |X[l, j]| < 2^e_j.  ecol is
// first set to kNoExp; a column that stays there is all zero.
constexpr int kNoExp = -100000;

__global__ void colexp_init_kernel(int* __restrict__ ecol, int64_t Q) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < Q) ecol[j] = kNoExp;
}

__global__ void colexp_kernel(const double* __restrict__ X, int64_t l0, int64_t l1, int64_t Q,
                              int64_t ldx, int64_t rows_per_block, int* __restrict__ ecol) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Q) return;
  const int64_t r0 = l0 + (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = min(l1, r0 + rows_per_block);
  double mx = 0.0;
  for (int64_t l = r0; l < r1; ++l) mx = fmax(mx, fabs(X[l * ldx + j]));
  if (mx > 0.0) {
    int e = 0;
    frexp(mx, &e);
    atomicMax(&ecol[j], e);
  }
}

__device__ __forceinline__ int col_exponent(const int* ecol, int64_t j) {
  const int e = ecol[j];
  return e == kNoExp ? 0 : e;
}

// The tensor-core GEMM over one segment: Cseg[i, j] += 2^(e_j - 11) * scale *
// sum_g 2^(-8 g) * sum_l (group g products).  Gt holds [Gh; Gl] and Dt the 8
// planes of X's digits, both as pre-swizzled tiles (tiled_off).  One thread
// issues the bulk copies and the MMAs: the K-tile k + 1 is loaded into the
// stage freed by the MMAs of k - 1 (tracked by mbarriers), so loads overlap
// the MMAs of k and the TMEM drain at the end of a chunk, which all eight
// warps share.
constexpr int TC_STAGE_TX = 2 * TILE_A_BYTES + TC_DIGITS * TILE_B_BYTES;

// One 128 x 64 output tile (rows i0.., columns j0.. of C) of one problem's
// digit planes: the body of sketch_tc_kernel and sketch_tc_grouped_kernel.
__device__ __forceinline__ void sketch_tc_tile(
    const uint16_t* __restrict__ Gt, const uint16_t* __restrict__ Dt, int64_t Sp, int64_t Qp,
    int64_t Lp, int64_t Kext, const int* __restrict__ ecol, double scale, int64_t S, int64_t Q,
    double* __restrict__ C, int64_t ldc, int* __restrict__ err, int64_t i0, int64_t j0) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + 2 * STAGE_BYTES);   // full[2], empty[2], done
  uint64_t* full = bars;
  uint64_t* empty = bars + 2;
  uint64_t* done = bars + 4;
  uint32_t* tmem_slot = (uint32_t*)(bars + 5);
  int* abort_flag = (int*)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    for (int q = 0; q < 5; ++q) mbar_init(&bars[q], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // The digit tiles d_1..d_8 lie back to back (64 rows of 128 bytes each), so
  // d_1..d_4 and d_5..d_8 are each one K-major 256-row operand: one MMA with
  // N = 256 covers four groups at once (TMEM column 64 g holds group g).
  constexpr uint32_t idesc256 = instr_desc(TC_M, 4 * TC_N);
  constexpr uint32_t idesc192 = instr_desc(TC_M, 3 * TC_N);

  // Exact column sums: group sums S_g (integers, |S_g| <= 2^24) of every chunk
  // go into two int64 accumulators per column,
  //   A1 += S_0 2^24 + S_1 2^16 + S_2 2^8 + S_3,  A2 += S_4 2^24 + ... + S_7,
  // each below 2^48.01 per chunk (safe for 2^14 chunks); the value is
  // A1 2^-24 + A2 2^-56.  Warpgroup h drains columns [32 h, 32 h + 32).
  const int wg = warp >> 2;
  long long a1[32], a2[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) a1[c] = a2[c] = 0;

  const int64_t nkt = Kext / TC_KT;   // K-tiles of this segment
  const int kt_per_chunk = TC_CHUNK / TC_KT;
  const int64_t nchunk = (nkt + kt_per_chunk - 1) / kt_per_chunk;
  int64_t issued = 0, consumed = 0;   // thread 0: tiles loaded / whose MMAs were issued
  auto issue = [&](int64_t k) {
    const int st = (int)(k & 1);
    unsigned char* sbase = smem + st * STAGE_BYTES;
    const uint32_t s_ah = smem_addr(sbase);
    const uint32_t s_al = s_ah + TILE_A_BYTES;
    const uint32_t s_d = s_al + TILE_A_BYTES;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&full[st])),
                 "r"(TC_STAGE_TX)
                 : "memory");
    const int64_t nkt_l = Lp / TC_KT;   // K-tiles per tile row of a plane
    bulk_g2s(s_ah, Gt + tiled_off(i0, k * TC_KT, TC_M, nkt_l), TILE_A_BYTES, &full[st]);
    bulk_g2s(s_al, Gt + Sp * Lp + tiled_off(i0, k * TC_KT, TC_M, nkt_l), TILE_A_BYTES, &full[st]);
#pragma unroll 1
    for (int p = 0; p < TC_DIGITS; ++p)
      bulk_g2s(s_d + p * TILE_B_BYTES, Dt + p * Qp * Lp + tiled_off(j0, k * TC_KT, TC_N, nkt_l),
               TILE_B_BYTES, &full[st]);
    issued = k + 1;
  };
  if (tid == 0) {
    if (nkt > 0) issue(0);
    if (nkt > 1) issue(1);
  }
  bool ok = true;
  for (int64_t ch = 0; ch < nchunk; ++ch) {
    const int64_t kt = ch * kt_per_chunk;
    const int64_t kt_end = (kt + kt_per_chunk < nkt) ? kt + kt_per_chunk : nkt;
    if (warp == 0) {
      if (tid == 0 && ok) {
      for (int64_t k = kt; k < kt_end; ++k) {
        const int st = (int)(k & 1);
        if (!mbar_wait(&full[st], (uint32_t)((k >> 1) & 1), err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // descriptors differ only in the start address field (address >> 4)
        const uint64_t d_ah = smem_desc(smem_addr(smem + st * STAGE_BYTES));
        const uint64_t d_al = d_ah + (TILE_A_BYTES >> 4);
        const uint64_t d_b = d_al + (TILE_A_BYTES >> 4);
        const uint64_t d_b5 = d_b + (uint64_t)(4 * (TILE_B_BYTES >> 4));
#pragma unroll
        for (int ks = 0; ks < TC_KT / 16; ++ks) {
          const uint32_t acc0 = (k == kt && ks == 0) ? 0u : 1u;
          // h d_{g+1} into groups 0-3 and 4-7 (these start a chunk's sums),
          // then g_lo d_g into groups 1-4 and 5-7 (g_lo d_8 is dropped)
          mma_bf16(tmem, d_ah + 2 * ks, d_b + 2 * ks, idesc256, acc0);
          mma_bf16(tmem + (uint32_t)(4 * TC_N), d_ah + 2 * ks, d_b5 + 2 * ks, idesc256, acc0);
          mma_bf16(tmem + (uint32_t)TC_N, d_al + 2 * ks, d_b + 2 * ks, idesc256, 1u);
          mma_bf16(tmem + (uint32_t)(5 * TC_N), d_al + 2 * ks, d_b5 + 2 * ks, idesc192, 1u);
        }
        mma_commit(&empty[st]);
        consumed = k + 1;
        if (k + 1 == kt_end) mma_commit(done);
        // refill the stage of k - 1 with tile k + 1 once the MMAs of k - 1 are done
        if (k >= 1 && k + 1 < nkt && issued == k + 1) {
          if (!mbar_wait(&empty[st ^ 1], (uint32_t)(((k - 1) >> 1) & 1), err)) {
            ok = false;
            break;
          }
          issue(k + 1);
        }
      }
      // the chunk's MMAs complete before any warp reads TMEM
      if (ok && !mbar_wait(done, (uint32_t)(ch & 1), err)) ok = false;
      if (!ok) *abort_flag = 1;
      }
      __syncwarp();   // the other lanes of warp 0 wait here, not in a spin loop
    }
    // every warp: the chunk's MMAs are complete (thread 0 saw `done`) -> drain TMEM
    __syncthreads();
    const bool have = *abort_flag == 0;
    tc_fence_after();
    if (have) {
      const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll 1
      for (int g = 0; g < 4; ++g) {
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(g * TC_N + wg * 32), v);
        const long long w = 1ll << (24 - 8 * g);
#pragma unroll
        for (int c = 0; c < 32; ++c) a1[c] += (long long)__float2int_rn(v[c]) * w;   // exact
      }
#pragma unroll 1
      for (int g = 4; g < TC_GROUPS; ++g) {
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(g * TC_N + wg * 32), v);
        const long long w = 1ll << (24 - 8 * (g - 4));
#pragma unroll
        for (int c = 0; c < 32; ++c) a2[c] += (long long)__float2int_rn(v[c]) * w;
      }
    } else {
      ok = false;
    }
    tc_fence_before();
    __syncthreads();   // TMEM may be overwritten by the next chunk's first MMAs
    if (*abort_flag != 0) {
      ok = false;
      break;
    }
  }
  if (tid == 0 && !ok) {
    // let issued copies and MMAs finish (bounded) before the CTA releases its memory
    for (int64_t k = consumed; k < issued; ++k) mbar_wait(&full[k & 1], (uint32_t)((k >> 1) & 1), err);
    for (int64_t k = consumed >= 2 ? consumed - 2 : 0; k < consumed; ++k)
      mbar_wait(&empty[k & 1], (uint32_t)((k >> 1) & 1), err);
  }
  // epilogue: row i0 + 32 (warp % 4) + lane, columns j0 + 32 wg .. + 31
  const int64_t i = i0 + (warp & 3) * 32 + (tid & 31);
  if (ok && i < S) {
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const int64_t j = j0 + wg * 32 + c;
      if (j < Q) {
        const double v = fma((double)a2[c], 0x1p-56, (double)a1[c] * 0x1p-24);
        C[i * ldc + j] += ldexp(v, col_exponent(ecol, j) - 11) * scale;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1) sketch_tc_kernel(
    const uint16_t* __restrict__ Gt, const uint16_t* __restrict__ Dt, int64_t Sp, int64_t Qp,
    int64_t Lp, int64_t Kext, const int* __restrict__ ecol, double scale, int64_t S, int64_t Q,
    double* __restrict__ C, int64_t ldc, int* __restrict__ err) {
  // row tiles vary fastest
  sketch_tc_tile(Gt, Dt, Sp, Qp, Lp, Kext, ecol, scale, S, Q, C, ldc, err,
                 (int64_t)blockIdx.x * TC_M, (int64_t)blockIdx.y * TC_N);
}

// Grouped sketch of several problems in one launch: CTA b runs tile tiles[b]
// = (problem, row tile, column tile) of the problem descriptors.
struct TcGroupDesc {
  const uint16_t* Gt;
  const uint16_t* Dt;
  int64_t Sp, Qp, Lp, Kext;
  const int* ecol;
  double scale;
  int64_t S, Q;
  double* C;
  int64_t ldc;
  int* err;
};

__global__ void __launch_bounds__(TC_THREADS, 1) sketch_tc_grouped_kernel(
    const TcGroupDesc* __restrict__ descs, const int4* __restrict__ tiles) {
  const int4 t = tiles[blockIdx.x];
  const TcGroupDesc d = descs[t.x];
  sketch_tc_tile(d.Gt, d.Dt, d.Sp, d.Qp, d.Lp, d.Kext, d.ecol, d.scale, d.S, d.Q, d.C, d.ldc, d.err,
                 (int64_t)t.y * TC_M, (int64_t)t.z * TC_N);
}

// Digit planes of X rows [l0, l0 + Ls): D[p][j][l - l0], transposed through shared memory.
// y = X 2^(7 - e_j) (|y| < 128) is formed exactly as the 64-bit fixed-point
// integer Y = y 2^56 (bits below 2^-56 are rounded off), and its balanced
// base-256 digits are cut with integer shifts: d_1 = round(Y / 2^56),
// Y -= d_1 2^56, d_2 = round(Y / 2^48), ..., d_8 = Y (|d_p| <= 128), so that
// y = sum_p d_p 2^(8 - 8p) up to the rounding of Y.  |Y| may come within
// 2^55 of 2^63, so rounding shifts before adding and the subtraction wraps.
__device__ __forceinline__ long long fixed56(double x, int ej) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0) return 0;                       // zero (and subnormals, below 2^-1022)
  long long mant = (long long)((bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = ex - 1075 - ej + 63;           // Y = mant 2^sh
  long long y;
  if (sh >= 0) y = mant * (1ll << sh);          // |Y| < 2^63 since |x| < 2^e_j
  else if (sh > -64) y = (mant + (1ll << (-sh - 1))) >> (-sh);
  else y = 0;
  return (bits >> 63) ? -y : y;
}

__global__ void __launch_bounds__(256) split_x_kernel(const double* __restrict__ X, int64_t l0,
                                                      int64_t l1, int64_t Q, int64_t ldx,
                                                      const int* __restrict__ ecol, int64_t Qp,
                                                      int64_t Lp, uint16_t* __restrict__ D) {
  __shared__ unsigned short tile[TC_DIGITS][32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const int64_t jb = (int64_t)blockIdx.x * 32, lb = (int64_t)blockIdx.y * 32;
  for (int r = ty; r < 32; r += 8) {
    const int64_t l = l0 + lb + r, j = jb + tx;
    long long y = 0;
    if (l < l1 && j < Q) y = fixed56(X[l * ldx + j], col_exponent(ecol, j));
#pragma unroll
    for (int p = 0; p < TC_DIGITS; ++p) {
      const int s = 56 - 8 * p;
      // round(y / 2^s) without forming y + 2^(s-1), which can exceed 2^63
      const long long d = s > 0 ? (((y >> (s - 1)) + 1) >> 1) : y;
      // |y - d 2^s| <= 2^(s-1): exact in modular arithmetic even when d 2^s = 2^63
      y = (long long)((unsigned long long)y - ((unsigned long long)d << s));
      tile[p][r][tx] = (unsigned short)(__float_as_uint(__int2float_rn((int)d)) >> 16);
    }
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t j = jb + r, l = lb + tx;
    if (j < Qp && l < Lp) {
#pragma unroll
      for (int p = 0; p < TC_DIGITS; ++p) {
        D[(int64_t)p * Qp * Lp + tiled_off(j, l, TC_N, Lp / TC_KT)] = tile[p][tx][r];
      }
    }
  }
}

// Digit planes of Gamma rows [l0, l0 + Ls): Gh[i][l - l0], Gl[i][l - l0].
__global__ void __launch_bounds__(256) gamma_digits_kernel(uint64_t seed, uint32_t tag, int64_t l0,
                                                           int64_t l1, int64_t S, int64_t Sp,
                                                           int64_t Lp,
                                                           uint16_t* __restrict__ Gh,
                                                           uint16_t* __restrict__ Gl, int64_t lbase) {
  __shared__ unsigned short th[32][129], tl[32][129];
  const int64_t ib = (int64_t)blockIdx.x * 128, lb = (int64_t)blockIdx.y * 32;
  // generate: thread -> (row r of 32, group of four sketch indices g4 of 32)
  for (int q = threadIdx.x; q < 32 * 32; q += 256) {
    const int r = q >> 5, g4 = q & 31;
    const int64_t l = l0 + lb + r;
    const int64_t i = ib + 4 * g4;
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (l < l1 && i < S) z = normal4(seed, tag, (uint64_t)(lbase + l), (uint64_t)(i >> 2));
    const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float qv = (l < l1 && i + k < S) ? rintf(__fmul_rn(zz[k], 4096.0f)) : 0.0f;
      qv = fminf(fmaxf(qv, -32767.0f), 32767.0f);
      const float h = rintf(qv * (1.0f / 256.0f));
      const float lo = qv - 256.0f * h;
      th[r][4 * g4 + k] = (unsigned short)(__float_as_uint(h) >> 16);
      tl[r][4 * g4 + k] = (unsigned short)(__float_as_uint(lo) >> 16);
    }
  }
  __syncthreads();
  // write: row i (128 of them), 32 consecutive l
  for (int q = threadIdx.x; q < 128 * 32; q += 256) {
    const int ii = q >> 5, r = q & 31;
    const int64_t i = ib + ii, l = lb + r;
    if (i < Sp && l < Lp) {
      Gh[tiled_off(i, l, TC_M, Lp / TC_KT)] = th[r][ii];
      Gl[tiled_off(i, l, TC_M, Lp / TC_KT)] = tl[r][ii];
    }
  }
}

__global__ void zero_kernel(double* __restrict__ C, int64_t S, int64_t Q, int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < S * Q) C[(idx / Q) * ldc + idx % Q] = 0.0;
}


// ---- single-pass BF16 sketch (sketch mode LSRN_SKETCH_BF16) -------------------
// C = Gamma^T X with both operands rounded to bf16 once (Gamma's 2^-12 grid
// value, and X / 2^e_j with a per-column exponent so any FP64 range fits) and
// FP32 accumulation on the tensor cores: a subspace embedding with relative
// error ~2^-8, for well-conditioned full-rank problems (see the AUTO mode).
// Tile 128 sketch rows x 256 columns of X; one CTA per tile and K split.
// Warp 0 streams K-tiles (16 KB of Gamma, 32 KB of X, pre-swizzled) into a
// four-stage ring with bulk copies; warp 1 issues the MMAs (M=128, N=256,
// K=16) into one of two TMEM accumulators (256 columns each), switching every
// 2048 rows; warps 2-9 drain a finished accumulator into FP32 registers while
// the MMAs fill the other, so FP32 rounding grows with 2048 rather than with
// the whole K range.  Each CTA writes its FP64 partial tile; a fixed-order
// reduction adds the K splits.
constexpr int BF_M = 128, BF_N = 256, BF_KT = 64, BF_STAGES = 4, BF_CHUNK_KT = 32;
constexpr int BF_A_BYTES = BF_M * BF_KT * 2;             // 16 KB
constexpr int BF_B_BYTES = BF_N * BF_KT * 2;             // 32 KB
constexpr int BF_STAGE_BYTES = BF_A_BYTES + BF_B_BYTES;  // 48 KB
constexpr int BF_THREADS = 320;
constexpr int BF_SMEM = BF_STAGES * BF_STAGE_BYTES + 1024 + 256;
constexpr uint64_t kBfWaitNs = 200000000ull;   // 0.2 s per wait
__device__ __forceinline__ bool bf_wait(uint64_t* bar, uint32_t parity, int* err) {
  return mbar_wait_ns(bar, parity, err, kBfWaitNs);
}

__global__ void __launch_bounds__(BF_THREADS, 1) sketch_bf16_kernel(
    const uint16_t* __restrict__ Gt, const uint16_t* __restrict__ Xt, int64_t Lp, int64_t nkt,
    int64_t kt_per_split, const int* __restrict__ ecol, int64_t S, int64_t Q,
    double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + BF_STAGES * BF_STAGE_BYTES);
  uint64_t* full = bars;                       // [BF_STAGES]
  uint64_t* empty = bars + BF_STAGES;          // [BF_STAGES]
  uint64_t* tfull = bars + 2 * BF_STAGES;      // [2] accumulator b holds a finished chunk
  uint64_t* tempty = tfull + 2;                // [2] accumulator b drained (8 warp arrivals)
  uint64_t* mdone = tempty + 2;                // all MMAs of this CTA complete
  uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* s_issued = (volatile int*)(tmem_slot + 2);
  volatile int* s_consumed = (volatile int*)(tmem_slot + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = (int64_t)blockIdx.x * BF_M;
  const int64_t j0 = (int64_t)blockIdx.y * BF_N;
  const int64_t kb = (int64_t)blockIdx.z * kt_per_split;
  const int64_t ke = min(nkt, kb + kt_per_split);
  const int nk = (int)max((int64_t)0, ke - kb);
  const int nchunks = (nk + BF_CHUNK_KT - 1) / BF_CHUNK_KT;
  const int64_t nkt_row = Lp / BF_KT;          // K-tiles per tile row of a plane

  if (tid == 0) {
    for (int q = 0; q < BF_STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    mbar_init(&tfull[0], 1);
    mbar_init(&tfull[1], 1);
    mbar_init(&tempty[0], 8);
    mbar_init(&tempty[1], 8);
    mbar_init(mdone, 1);
    *abort_flag = 0;
    *s_issued = 0;
    *s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      for (int k = 0; k < nk && !*abort_flag; ++k) {
        const int st = k % BF_STAGES, n = k / BF_STAGES;
        if (n >= 1 && !bf_wait(&empty[st], (uint32_t)((n - 1) & 1), err)) {
          *abort_flag = 1;
          break;
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         smem_addr(&full[st])),
                     "r"(BF_STAGE_BYTES)
                     : "memory");
        const uint32_t sa = smem_addr(smem + st * BF_STAGE_BYTES);
        const int64_t kt = kb + k;
        bulk_g2s(sa, Gt + tiled_off(i0, kt * BF_KT, BF_M, nkt_row), BF_A_BYTES, &full[st]);
        bulk_g2s(sa + BF_A_BYTES, Xt + tiled_off(j0, kt * BF_KT, BF_N, nkt_row), BF_B_BYTES,
                 &full[st]);
        *s_issued = k + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = instr_desc(BF_M, BF_N);
      for (int k = 0; k < nk && !*abort_flag; ++k) {
        const int c = k / BF_CHUNK_KT, b = c & 1;
        const bool first = (k % BF_CHUNK_KT) == 0;
        if (first && c >= 2 && !bf_wait(&tempty[b], (uint32_t)(((c >> 1) - 1) & 1), err)) {
          *abort_flag = 1;
          break;
        }
        const int st = k % BF_STAGES;
        if (!bf_wait(&full[st], (uint32_t)((k / BF_STAGES) & 1), err)) {
          *abort_flag = 1;
          break;
        }
        *s_consumed = k + 1;
        tc_fence_after();
        const uint64_t da = smem_desc(smem_addr(smem + st * BF_STAGE_BYTES));
        const uint64_t db = da + (BF_A_BYTES >> 4);
#pragma unroll
        for (int ks = 0; ks < BF_KT / 16; ++ks)
          mma_bf16(tmem + (uint32_t)(b * BF_N), da + 2 * ks, db + 2 * ks, idesc,
                   (first && ks == 0) ? 0u : 1u);
        mma_commit(&empty[st]);
        if ((k % BF_CHUNK_KT) == BF_CHUNK_KT - 1 || k == nk - 1) mma_commit(&tfull[b]);
      }
      // every MMA issued above completes before the CTA frees TMEM or exits
      mma_commit(mdone);
      bf_wait(mdone, 0u, err);
    }
    __syncwarp();
  } else {
    // warps 2..9: TMEM lane quadrant warp % 4, columns [128 h, 128 h + 128), h = (warp - 2) / 4
    const int quad = warp & 3, h = (warp - 2) >> 2;
    float acc[128];
#pragma unroll
    for (int t = 0; t < 128; ++t) acc[t] = 0.0f;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1;
      bool ok = true;
      if (lane == 0) ok = bf_wait(&tfull[b], (uint32_t)((c >> 1) & 1), err);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok || *abort_flag) {
        if (lane == 0) *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * BF_N + h * 128);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float v[32];
        tmem_ld32(base + (uint32_t)(g * 32), v);
#pragma unroll
        for (int t = 0; t < 32; ++t) acc[g * 32 + t] += v[t];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&tempty[b])) : "memory");
    }
    const int64_t i = i0 + quad * 32 + lane;
    if (i < S && !*abort_flag) {
      double* out = part + (int64_t)blockIdx.z * S * Q + i * Q;
#pragma unroll
      for (int t = 0; t < 128; ++t) {
        const int64_t j = j0 + h * 128 + t;
        if (j < Q) out[j] = ldexp((double)acc[t], col_exponent(ecol, j));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) {
    atomicExch(err, 1);
    // copies issued but never consumed must land before the CTA's memory is released
    for (int k = *s_consumed; k < *s_issued; ++k)
      bf_wait(&full[k % BF_STAGES], (uint32_t)((k / BF_STAGES) & 1), err);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// bf16 tiles of X rows [l0, l1) scaled by 2^-e_j: D[tiled_off(j, l - l0, 256, Lp / 64)]
__global__ void __launch_bounds__(256) x_bf16_kernel(const double* __restrict__ X, int64_t l0,
                                                     int64_t l1, int64_t Q, int64_t ldx,
                                                     const int* __restrict__ ecol, int64_t Qp,
                                                     int64_t Lp, uint16_t* __restrict__ D) {
  __shared__ unsigned short tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t jb = (int64_t)blockIdx.x * 32, lb = (int64_t)blockIdx.y * 32;
  for (int r = ty; r < 32; r += 8) {
    const int64_t l = l0 + lb + r, j = jb + tx;
    unsigned short v = 0;
    if (l < l1 && j < Q) {
      const __nv_bfloat16 bv = __double2bfloat16(ldexp(X[l * ldx + j], -col_exponent(ecol, j)));
      v = *reinterpret_cast<const unsigned short*>(&bv);
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t j = jb + r, l = lb + tx;
    if (j < Qp && l < Lp) D[tiled_off(j, l, BF_N, Lp / BF_KT)] = tile[tx][r];
  }
}

// bf16 tiles of Gamma rows [l0, l1): G[tiled_off(i, l - l0, 128, Lp / 64)] = bf16(Gamma[l, i])
__global__ void __launch_bounds__(256) gamma_bf16_kernel(uint64_t seed, uint32_t tag, int64_t l0,
                                                         int64_t l1, int64_t S, int64_t Sp, int64_t Lp,
                                                         uint16_t* __restrict__ G, int64_t lbase) {
  __shared__ unsigned short tg[32][129];
  const int64_t ib = (int64_t)blockIdx.x * 128, lb = (int64_t)blockIdx.y * 32;
  for (int q = threadIdx.x; q < 32 * 32; q += 256) {
    const int r = q >> 5, g4 = q & 31;
    const int64_t l = l0 + lb + r;
    const int64_t i = ib + 4 * g4;
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (l < l1 && i < S) z = normal4(seed, tag, (uint64_t)(lbase + l), (uint64_t)(i >> 2));
    const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float g = (l < l1 && i + k < S) ? quantize_g(zz[k]) : 0.0f;
      const __nv_bfloat16 bv = __float2bfloat16_rn(g);
      tg[r][4 * g4 + k] = *reinterpret_cast<const unsigned short*>(&bv);
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 128 * 32; q += 256) {
    const int ii = q >> 5, r = q & 31;
    const int64_t i = ib + ii, l = lb + r;
    if (i < Sp && l < Lp) G[tiled_off(i, l, BF_M, Lp / BF_KT)] = tg[r][ii];
  }
}

// C[i, j] += scale * sum_z part[z][i, j], z in order
__global__ void bf16_reduce_kernel(const double* __restrict__ part, int nz, int64_t S, int64_t Q,
                                   double scale, double* __restrict__ C, int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * Q) return;
  double acc = 0.0;
  for (int z = 0; z < nz; ++z) acc += part[(int64_t)z * S * Q + idx];
  C[(idx / Q) * ldc + idx % Q] += scale * acc;
}

// K split of the BF16 sketch: the smallest split whose CTA count fills whole
// waves of one CTA per SM to >= 95%, else the best of at most 64.
int bf16_ksplit(int64_t tiles, int64_t nkt) {
  const int64_t sms = num_sms();
  int best = 1;
  double best_eff = 0.0;
  for (int z = 1; z <= 64 && z <= std::max<int64_t>(1, nkt / 8); ++z) {
    const int64_t ctas = tiles * z;
    const int64_t waves = (ctas + sms - 1) / sms;
    const double eff = (double)ctas / (double)(waves * sms);
    if (eff >= 0.95) return z;
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = z;
    }
  }
  return best;
}
}  // namespace

// Scratch bytes for a given segment length (rows of X per segment).
size_t sketch_tc_scratch_bytes(int64_t Ls, int64_t Q, int64_t S) {
  const int64_t Lp = (Ls + TC_KT - 1) / TC_KT * TC_KT;
  const int64_t Qp = (Q + TC_N - 1) / TC_N * TC_N;
  const int64_t Sp = (S + TC_M - 1) / TC_M * TC_M;
  return (size_t)(2 * Sp + TC_DIGITS * Qp) * Lp * 2 + (size_t)Q * sizeof(int) + 256;
}

int64_t sketch_tc_segment_rows(int64_t L, int64_t Q, int64_t S, size_t budget_bytes) {
  const int64_t Qp = (Q + TC_N - 1) / TC_N * TC_N;
  const int64_t Sp = (S + TC_M - 1) / TC_M * TC_M;
  const int64_t per_row = (2 * Sp + TC_DIGITS * Qp) * 2;
  int64_t rows = (int64_t)(budget_bytes / (size_t)std::max<int64_t>(per_row, 1));
  rows = std::max<int64_t>(TC_CHUNK, rows / TC_CHUNK * TC_CHUNK);
  rows = std::min<int64_t>(rows, (int64_t)8192 * TC_CHUNK);   // int64 column sums stay exact
  const int64_t Lr = (L + TC_KT - 1) / TC_KT * TC_KT;
  return std::min(rows, Lr);
}

lsrn_status launch_sketch_tc(const double* X, int64_t L, int64_t Q, int64_t ldx, double xscale,
                             int64_t S, uint64_t seed, uint32_t tag, double* C, int64_t ldc,
                             void* scratch, size_t scratch_bytes, int64_t seg_rows, int* err,
                             cudaStream_t st,
                             std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* gemm_events,
                             int64_t lbase) {
  const int64_t Qp = (Q + TC_N - 1) / TC_N * TC_N;
  const int64_t Sp = (S + TC_M - 1) / TC_M * TC_M;
  const int64_t Lp = (seg_rows + TC_KT - 1) / TC_KT * TC_KT;
  if (scratch_bytes < sketch_tc_scratch_bytes(seg_rows, Q, S)) return LSRN_ERR_INVALID_ARG;
  LSRN_CUDA_TRY(cudaFuncSetAttribute(sketch_tc_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  uint16_t* Gh = (uint16_t*)scratch;
  uint16_t* Gl = Gh + Sp * Lp;
  uint16_t* D = Gl + Sp * Lp;
  int* ecol = (int*)(D + (int64_t)TC_DIGITS * Qp * Lp);
  const int64_t tot = S * Q;
  launch(zero_kernel, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, st, C, S, Q, ldc);
  for (int64_t l0 = 0; l0 < L; l0 += seg_rows) {
    const int64_t l1 = std::min(L, l0 + seg_rows);
    const int64_t Lseg = (l1 - l0 + TC_KT - 1) / TC_KT * TC_KT;   // K extent streamed
    const int64_t rpb = 1024;
    launch(colexp_init_kernel, dim3((unsigned)((Q + 255) / 256)), dim3(256), 0, st, ecol, Q);
    launch(colexp_kernel, dim3((unsigned)((Q + 127) / 128), (unsigned)((l1 - l0 + rpb - 1) / rpb)),
           dim3(128), 0, st, X, l0, l1, Q, ldx, rpb, ecol);
    launch(split_x_kernel, dim3((unsigned)(Qp / 32), (unsigned)(Lp / 32)), dim3(256), 0, st, X, l0,
           l1, Q, ldx, (const int*)ecol, Qp, Lp, D);
    launch(gamma_digits_kernel, dim3((unsigned)(Sp / 128), (unsigned)(Lp / 32)), dim3(256), 0, st,
           seed, tag, l0, l1, S, Sp, Lp, Gh, Gl, lbase);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (gemm_events) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, st);
    }
    // the column tiles that share an X digit tile run together (y fastest):
    // the smaller Gamma planes are the ones re-read across waves
    launch(sketch_tc_kernel, dim3((unsigned)(Sp / TC_M), (unsigned)(Qp / TC_N)), dim3(TC_THREADS),
           (size_t)TC_SMEM, st, (const uint16_t*)Gh, (const uint16_t*)D, Sp, Qp, Lp, Lseg,
           (const int*)ecol, xscale, S, Q, C, ldc, err);
    if (gemm_events) {
      cudaEventRecord(e1, st);
      gemm_events->emplace_back(e0, e1);
    }
  }
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}


static size_t tc_round256(size_t b) { return (b + 255) / 256 * 256; }

size_t sketch_tc_group_scratch_bytes(const std::vector<TcGroupItem>& items) {
  size_t b = 0, tiles = 0;
  for (const TcGroupItem& it : items) {
    b += tc_round256(sketch_tc_scratch_bytes(it.L, it.Q, it.S));
    tiles += (size_t)((it.S + TC_M - 1) / TC_M) * (size_t)((it.Q + TC_N - 1) / TC_N);
  }
  return b + tc_round256(items.size() * sizeof(TcGroupDesc)) + tc_round256(tiles * sizeof(int4));
}

lsrn_status launch_sketch_tc_grouped(const std::vector<TcGroupItem>& items, void* scratch,
                                     size_t scratch_bytes, cudaStream_t st) {
  if (items.empty()) return LSRN_OK;
  if (scratch_bytes < sketch_tc_group_scratch_bytes(items)) return LSRN_ERR_INVALID_ARG;
  LSRN_CUDA_TRY(cudaFuncSetAttribute(sketch_tc_grouped_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  unsigned char* base = (unsigned char*)scratch;
  std::vector<TcGroupDesc> descs;
  std::vector<int64_t> klen;
  for (const TcGroupItem& it : items) {
    // the single segment of launch_sketch_tc, planes in this problem's slice
    const int64_t Qp = (it.Q + TC_N - 1) / TC_N * TC_N;
    const int64_t Sp = (it.S + TC_M - 1) / TC_M * TC_M;
    const int64_t Lp = (it.L + TC_KT - 1) / TC_KT * TC_KT;
    uint16_t* Gh = (uint16_t*)base;
    uint16_t* Gl = Gh + Sp * Lp;
    uint16_t* D = Gl + Sp * Lp;
    int* ecol = (int*)(D + (int64_t)TC_DIGITS * Qp * Lp);
    base += tc_round256(sketch_tc_scratch_bytes(it.L, it.Q, it.S));
    const int64_t tot = it.S * it.Q;
    const int64_t rpb = 1024;
    launch(zero_kernel, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, st, it.C, it.S, it.Q, it.ldc);
    launch(colexp_init_kernel, dim3((unsigned)((it.Q + 255) / 256)), dim3(256), 0, st, ecol, it.Q);
    launch(colexp_kernel, dim3((unsigned)((it.Q + 127) / 128), (unsigned)((it.L + rpb - 1) / rpb)),
           dim3(128), 0, st, it.X, (int64_t)0, it.L, it.Q, it.ldx, rpb, ecol);
    launch(split_x_kernel, dim3((unsigned)(Qp / 32), (unsigned)(Lp / 32)), dim3(256), 0, st, it.X,
           (int64_t)0, it.L, it.Q, it.ldx, (const int*)ecol, Qp, Lp, D);
    launch(gamma_digits_kernel, dim3((unsigned)(Sp / 128), (unsigned)(Lp / 32)), dim3(256), 0, st,
           it.seed, it.tag, (int64_t)0, it.L, it.S, Sp, Lp, Gh, Gl, it.lbase);
    descs.push_back(TcGroupDesc{Gh, D, Sp, Qp, Lp, Lp, ecol, it.xscale, it.S, it.Q, it.C, it.ldc, it.err});
    klen.push_back(Lp);
  }
  // tiles of the longest problems first (a tile's time grows with its K extent);
  // within a problem the row tiles vary fastest, as in the single launch
  std::vector<int> order(items.size());
  for (size_t k = 0; k < items.size(); ++k) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return klen[a] > klen[b]; });
  std::vector<int4> tiles;
  for (int k : order)
    for (int64_t tj = 0; tj < descs[k].Qp / TC_N; ++tj)
      for (int64_t ti = 0; ti < descs[k].Sp / TC_M; ++ti) tiles.push_back(make_int4(k, (int)ti, (int)tj, 0));
  TcGroupDesc* ddesc = (TcGroupDesc*)base;
  base += tc_round256(descs.size() * sizeof(TcGroupDesc));
  int4* dtiles = (int4*)base;
  LSRN_CUDA_TRY(cudaMemcpyAsync(ddesc, descs.data(), descs.size() * sizeof(TcGroupDesc),
                                cudaMemcpyHostToDevice, st));
  LSRN_CUDA_TRY(cudaMemcpyAsync(dtiles, tiles.data(), tiles.size() * sizeof(int4),
                                cudaMemcpyHostToDevice, st));
  launch(sketch_tc_grouped_kernel, dim3((unsigned)tiles.size()), dim3(TC_THREADS), (size_t)TC_SMEM, st,
         (const TcGroupDesc*)ddesc, (const int4*)dtiles);
  LSRN_CUDA_TRY(cudaGetLastError());
  // the host vectors must outlive the copies from pageable memory
  LSRN_CUDA_TRY(cudaStreamSynchronize(st));
  return LSRN_OK;
}

// ---- BF16 sketch launcher -----------------------------------------------------
static int64_t bf16_dims_Sp(int64_t S) { return (S + BF_M - 1) / BF_M * BF_M; }
static int64_t bf16_dims_Qp(int64_t Q) { return (Q + BF_N - 1) / BF_N * BF_N; }
// K splits of a segment of nkt K-tiles: bf16_ksplit, with the FP64 partial
// tiles (one S x Q copy per split) held to 1 GiB.
static int bf16_split_for(int64_t S, int64_t Q, int64_t nkt) {
  const int64_t tiles = (bf16_dims_Sp(S) / BF_M) * (bf16_dims_Qp(Q) / BF_N);
  const int64_t cap = std::max<int64_t>(1, ((int64_t)1 << 30) / std::max<int64_t>(1, S * Q * 8));
  return (int)std::min<int64_t>(bf16_ksplit(tiles, nkt), cap);
}

size_t sketch_bf16_scratch_bytes(int64_t Ls, int64_t Q, int64_t S) {
  const int64_t Lp = (Ls + BF_KT - 1) / BF_KT * BF_KT;
  return (size_t)(bf16_dims_Sp(S) + bf16_dims_Qp(Q)) * Lp * 2 + (size_t)Q * sizeof(int) + 256 +
         (size_t)bf16_split_for(S, Q, Lp / BF_KT) * S * Q * sizeof(double);
}

int64_t sketch_bf16_segment_rows(int64_t L, int64_t Q, int64_t S, size_t budget_bytes) {
  const size_t fixed = ((size_t)1 << 30) + (size_t)Q * 4 + 256;
  const int64_t per_row = (bf16_dims_Sp(S) + bf16_dims_Qp(Q)) * 2;
  const size_t room = budget_bytes > fixed ? budget_bytes - fixed : (size_t)per_row * BF_KT;
  int64_t rows = (int64_t)(room / (size_t)per_row);
  rows = std::max<int64_t>(BF_KT, rows / BF_KT * BF_KT);
  const int64_t Lr = (L + BF_KT - 1) / BF_KT * BF_KT;
  return std::min(rows, Lr);
}

lsrn_status launch_sketch_bf16(const double* X, int64_t L, int64_t Q, int64_t ldx, double xscale,
                               int64_t S, uint64_t seed, uint32_t tag, double* C, int64_t ldc,
                               void* scratch, size_t scratch_bytes, int64_t seg_rows, int* err,
                               cudaStream_t st,
                               std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* gemm_events,
                               int64_t lbase) {
  const int64_t Sp = bf16_dims_Sp(S), Qp = bf16_dims_Qp(Q);
  const int64_t Lp = (seg_rows + BF_KT - 1) / BF_KT * BF_KT;
  if (scratch_bytes < sketch_bf16_scratch_bytes(seg_rows, Q, S)) return LSRN_ERR_INVALID_ARG;
  LSRN_CUDA_TRY(cudaFuncSetAttribute(sketch_bf16_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, BF_SMEM));
  uint16_t* Gt = (uint16_t*)scratch;
  uint16_t* Xt = Gt + Sp * Lp;
  int* ecol = (int*)(Xt + Qp * Lp);
  double* part = (double*)(((uintptr_t)(ecol + Q) + 255) & ~(uintptr_t)255);
  const int64_t tot = S * Q;
  launch(zero_kernel, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, st, C, S, Q, ldc);
  for (int64_t l0 = 0; l0 < L; l0 += seg_rows) {
    const int64_t l1 = std::min(L, l0 + seg_rows);
    const int64_t nkt = (l1 - l0 + BF_KT - 1) / BF_KT;
    const int64_t rpb = 1024;
    launch(colexp_init_kernel, dim3((unsigned)((Q + 255) / 256)), dim3(256), 0, st, ecol, Q);
    launch(colexp_kernel, dim3((unsigned)((Q + 127) / 128), (unsigned)((l1 - l0 + rpb - 1) / rpb)),
           dim3(128), 0, st, X, l0, l1, Q, ldx, rpb, ecol);
    launch(x_bf16_kernel, dim3((unsigned)(Qp / 32), (unsigned)(Lp / 32)), dim3(256), 0, st, X, l0, l1,
           Q, ldx, (const int*)ecol, Qp, Lp, Xt);
    launch(gamma_bf16_kernel, dim3((unsigned)(Sp / 128), (unsigned)(Lp / 32)), dim3(256), 0, st,
           seed, tag, l0, l1, S, Sp, Lp, Gt, lbase);
    const int z = bf16_split_for(S, Q, nkt);
    const int64_t per = (nkt + z - 1) / z;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (gemm_events) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, st);
    }
    launch(sketch_bf16_kernel, dim3((unsigned)(Sp / BF_M), (unsigned)(Qp / BF_N), (unsigned)z),
           dim3(BF_THREADS), (size_t)BF_SMEM, st, (const uint16_t*)Gt, (const uint16_t*)Xt, Lp, nkt,
           per, (const int*)ecol, S, Q, part, err);
    if (gemm_events) {
      cudaEventRecord(e1, st);
      gemm_events->emplace_back(e0, e1);
    }
    launch(bf16_reduce_kernel, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, st,
           (const double*)part, z, S, Q, xscale, C, ldc);
  }
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

}  // namespace lsrn
