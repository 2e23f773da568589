// Split-precision (bf16x3) GEMM on the sm_103a tensor cores.
//
// C(m, n) = sum_k A(m, k) B(n, k) for fp64 data split as a = hi + lo with
// hi = bf16(a) and lo = bf16(a - hi):  C = A_hi B_hi + A_hi B_lo + A_lo B_hi,
// accumulated in FP32 in tensor memory (TMEM).  The dropped A_lo B_lo term
// and the bf16 rounding of lo bound the relative error of each product near
// 2^-16.
//
// Persistent kernel: one CTA per SM walks the 128 x BN output tiles (BN = 256
// or 128) t = blockIdx.x, blockIdx.x + gridDim.x, ... with 192 threads:
//   warp 0 lane 0  - TMA producer: per K block (64 wide, 128-byte swizzle;
//                    32 wide with 64-byte swizzle for the 128 x 256 two-plane
//                    tiles) it loads the operand tiles (A_hi, A_lo, B_hi,
//                    B_lo) with cp.async.bulk.tensor into a STAGES-deep ring,
//                    signalling a "full" mbarrier; the ring runs on across
//                    tile boundaries;
//   warp 1 lane 0  - MMA issuer: waits for "full", issues (K block / 16) x 3
//                    tcgen05.mma.kind::f16 (M=128, N=BN, K=16) into one of two
//                    TMEM accumulators (tiles alternate between them; the
//                    six-product GEMMs instead spread a tile's K blocks over
//                    four accumulators), releases each stage with
//                    tcgen05.commit on its "empty" mbarrier and the finished
//                    tile on an "acc full" mbarrier;
//   warps 2-5      - epilogue: tcgen05.ld 32x32b rows of the finished
//                    accumulator (warp w reads TMEM lanes 32 (w mod 4) ..),
//                    stores them (fp32 or fp64) with bounds checks, or mixes
//                    them with the MPO matrix (MIX), and hands the
//                    accumulator back ("acc empty"), so that the epilogue of
//                    one tile runs under the MMAs of the next.
// Every mbarrier wait is bounded (SEEMPS_WAIT_CLOCKS); a wait that runs out
// records SEEMPS_ERR_TIMEOUT, skips the remaining work, waits (bounded) for
// the copies and MMAs it issued and frees the TMEM before returning.
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "timing.cuh"

namespace {

constexpr int BM = 128;
constexpr int BK = 64;  // 64 bf16 = 128 bytes = one swizzle row

// NS bf16 planes per operand: 2 (hi, lo: bf16x3, 3 products) or 3 (hi, mid,
// lo: bf16x6, 6 products, used by the environment updates).
template <int BN, int NS>
struct TileCfg {
  static_assert(NS == 2 || (NS == 3 && BN == 128), "three planes only with 128-wide tiles");
  // K block of a pipeline stage: 32 for the 128 x 256 two-plane tiles (four
  // stages of 48 KB keep three stages of loads in flight), else 64
  static constexpr int BKT = (BN == 256 && NS == 2) ? 32 : 64;
  static constexpr int STAGES = BKT == 32 ? 4 : ((BN == 256 || NS == 3) ? 2 : 3);
  static constexpr int A_BYTES = BM * BKT * 2;
  static constexpr int B_BYTES = BN * BKT * 2;
  static constexpr int STAGE_BYTES = NS * A_BYTES + NS * B_BYTES;
  // per epilogue warp a padded 32 x 32 fp32 tile (together: the 128 x 32
  // chunk of the fused mixing), then the mixing matrix (<= 32 x 32 pairs
  // (w, w) of fp32) and its output offsets
  static constexpr int EPI_BYTES = 4 * 32 * 33 * 4 + 32 * 32 * 8 + 32 * 8;
  // TMEM: NBUF tile buffers of NACC accumulators (BN columns each).  The
  // two-plane GEMMs alternate tiles between two buffers; the six-product
  // GEMMs spread the K blocks of a tile over four accumulators (K block kb
  // into accumulator kb mod 4), which shortens each FP32 accumulation chain
  // in the tensor cores fourfold; the epilogue adds them in a fixed order.
  static constexpr int NACC = NS == 3 ? 4 : 1;
  static constexpr int NBUF = NS == 3 ? 1 : 2;
  static constexpr int TMEM_COLS = NACC * NBUF * BN;
  static_assert(TMEM_COLS <= 512, "TMEM columns");
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_BYTES + 1024 + 256;
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > SEEMPS_WAIT_CLOCKS) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
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

// Shared-memory matrix descriptor of a K-major tile written by TMA with
// rows of BKT bf16 swizzled over their width: BKT = 64 (128-byte rows,
// 128-byte swizzle, mode 2) or 32 (64-byte rows, 64-byte swizzle, mode 4);
// 8-row core groups stacked every 8 rows (stride byte offset), leading byte
// offset unused for these layouts, descriptor version 1 (bit 46).
template <int BKT>
__device__ __forceinline__ uint64_t sdesc_k(uint32_t saddr) {
  static_assert(BKT == 64 || BKT == 32, "K block");
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)((8u * BKT * 2u) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(BKT == 64 ? 2 : 4) << 61;
  return d;
}

// Instruction descriptor of tcgen05.mma.kind::f16: D fp32 (bits 4-5 = 1),
// A and B bf16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns: thread t of the warp receives
// lane (base lane + t), columns col .. col+31.
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void store_out(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_out(double* p, float v) { *p = (double)v; }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Output tile t of the persistent schedule: N tiles fastest, then M tiles,
// then the K split (z).
struct TileIdx {
  int m0, nt, kb0, nk, z;  // first row, N tile index, first K block, K blocks, split index
};

__device__ __forceinline__ TileIdx tile_of(int t, int tiles_n, int tiles_mn, int nk_all, int per_z, int bmu) {
  TileIdx r;
  r.z = t / tiles_mn;
  const int q = t - r.z * tiles_mn;
  r.m0 = (q / tiles_n) * bmu;
  r.nt = q % tiles_n;
  r.kb0 = r.z * per_z;
  r.nk = (nk_all - r.kb0) < per_z ? (nk_all - r.kb0) : per_z;
  return r;
}

__device__ __forceinline__ void epi_sync() {  // the four epilogue warps only
  asm volatile("bar.sync 1, 128;" ::: "memory");
}

// MIX: the epilogue applies the MPO mixing (MixEpi) instead of storing C;
// M tiles then start every bmu = apt Dl rows.
template <int BN, typename OutT, int NS, bool MIX>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_bf16x3_kernel(const __grid_constant__ CUtensorMap tAh,
                          const __grid_constant__ CUtensorMap tAl,
                          const __grid_constant__ CUtensorMap tAl2,
                          const __grid_constant__ CUtensorMap tBh,
                          const __grid_constant__ CUtensorMap tBl,
                          const __grid_constant__ CUtensorMap tBl2, OutT* __restrict__ C, int M,
                          int N, int Kp, ll ldc, int ksplit, int bmu, MixEpi mx, int* status,
                          const int* skip) {
  if (skip && *(volatile const int*)skip) return;  // uniform: before any barrier or TMEM use
  using Cfg = TileCfg<BN, NS>;
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* epi = reinterpret_cast<float*>(smem + STAGES * Cfg::STAGE_BYTES);
  uint64_t* full = (uint64_t*)(smem + STAGES * Cfg::STAGE_BYTES + Cfg::EPI_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // [2]: accumulator b holds a finished tile
  uint64_t* acce = accf + 2;        // [2]: the epilogue has drained accumulator b
  uint64_t* done = acce + 2;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = (N + BN - 1) / BN, tiles_mn = tiles_n * ((M + bmu - 1) / bmu);
  const int ntiles = tiles_mn * ksplit;
  // split K (ksplit > 1): tile z sums the K blocks [kb0, kb0 + nk) into its
  // own FP32 partial product, stored at C + z M ldc
  // split boundaries on 64-element K blocks whatever the stage's K block,
  // so that every tile shape forms the same partial sums
  const int nk_all = Kp / Cfg::BKT;
  const int per_z = ((Kp / BK + ksplit - 1) / ksplit) * (BK / Cfg::BKT);

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < Cfg::NBUF; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);  // one arrival per epilogue warp
    }
    mbar_init(done, 1);
    fence_mbar_init();
    prefetch_tmap(&tAh);
    prefetch_tmap(&tAl);
    prefetch_tmap(&tBh);
    prefetch_tmap(&tBl);
    if (NS == 3) {
      prefetch_tmap(&tAl2);
      prefetch_tmap(&tBl2);
    }
  }
  if (warp == 1) tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto stage_ptr = [&](int s, int which) -> uint8_t* {
    // which: 0 .. NS-1 the A planes (hi, lo[, lo2]), NS .. 2 NS - 1 the B planes
    uint8_t* base = smem + s * Cfg::STAGE_BYTES;
    if (which < NS) return base + which * Cfg::A_BYTES;
    return base + NS * Cfg::A_BYTES + (which - NS) * Cfg::B_BYTES;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: one ring over all K blocks of all tiles
      int g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TileIdx ti = tile_of(t, tiles_n, tiles_mn, nk_all, per_z, bmu);
        const int m0 = ti.m0, n0 = ti.nt * BN;
        for (int kb = 0; kb < ti.nk; ++kb, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)((g / STAGES) & 1);
          if ((g >= STAGES && !mbar_wait(&empty[s], ph ^ 1u)) || *(volatile int*)&s_fail) {
            atomicExch(&s_fail, 1);
            ok = false;
            break;
          }
          const int kx = (ti.kb0 + kb) * Cfg::BKT;
          mbar_arrive_expect_tx(&full[s], Cfg::STAGE_BYTES);
          tma_load_2d(stage_ptr(s, 0), &tAh, kx, m0, &full[s]);
          tma_load_2d(stage_ptr(s, 1), &tAl, kx, m0, &full[s]);
          if (NS == 3) tma_load_2d(stage_ptr(s, 2), &tAl2, kx, m0, &full[s]);
          tma_load_2d(stage_ptr(s, NS), &tBh, kx, n0, &full[s]);
          tma_load_2d(stage_ptr(s, NS + 1), &tBl, kx, n0, &full[s]);
          if (NS == 3) tma_load_2d(stage_ptr(s, NS + 2), &tBl2, kx, n0, &full[s]);
        }
      }
      // drain: the last min(STAGES, g) loads must have landed before the CTA
      // may exit (bounded; on a clean run these waits return at once)
      for (int q = (g > STAGES ? g - STAGES : 0); q < g; ++q) {
        if (!mbar_wait(&full[q % STAGES], (uint32_t)((q / STAGES) & 1))) atomicExch(&s_fail, 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
      int g = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const TileIdx ti = tile_of(t, tiles_n, tiles_mn, nk_all, per_z, bmu);
        const int b = i % Cfg::NBUF, use = i / Cfg::NBUF;
        // the buffer's previous tile (use - 1) must have been read out
        if (use > 0 && !mbar_wait(&acce[b], (uint32_t)((use - 1) & 1))) {
          atomicExch(&s_fail, 1);
          break;
        }
        tc_fence_after();
        for (int kb = 0; kb < ti.nk; ++kb, ++g) {
          const uint32_t d = tmem + (uint32_t)((b * Cfg::NACC + kb % Cfg::NACC) * BN);
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)((g / STAGES) & 1);
          if (!mbar_wait(&full[s], ph) || *(volatile int*)&s_fail) {
            atomicExch(&s_fail, 1);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = smem_u32(stage_ptr(s, 0)), al = smem_u32(stage_ptr(s, 1));
          const uint32_t bh = smem_u32(stage_ptr(s, NS)), bl = smem_u32(stage_ptr(s, NS + 1));
#pragma unroll
          for (int k = 0; k < Cfg::BKT / 16; ++k) {
            const uint32_t off = (uint32_t)(k * 32);  // 16 bf16 = 32 bytes along K
            const uint64_t dah = sdesc_k<Cfg::BKT>(ah + off), dal = sdesc_k<Cfg::BKT>(al + off);
            const uint64_t dbh = sdesc_k<Cfg::BKT>(bh + off), dbl = sdesc_k<Cfg::BKT>(bl + off);
            mma_bf16(d, dah, dbh, idesc, (kb >= Cfg::NACC || k != 0) ? 1u : 0u);
            mma_bf16(d, dah, dbl, idesc, 1u);
            mma_bf16(d, dal, dbh, idesc, 1u);
            if (NS == 3) {
              // the 2^-16 products: hi x lo2, mid x mid, lo2 x hi
              const uint64_t da2 = sdesc_k<Cfg::BKT>(smem_u32(stage_ptr(s, 2)) + off);
              const uint64_t db2 = sdesc_k<Cfg::BKT>(smem_u32(stage_ptr(s, NS + 2)) + off);
              mma_bf16(d, dah, db2, idesc, 1u);
              mma_bf16(d, dal, dbl, idesc, 1u);
              mma_bf16(d, da2, dbh, idesc, 1u);
            }
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&accf[b]);
      }
      // every MMA issued by this thread has completed before TMEM is freed
      mma_commit(done);
      if (!mbar_wait(done, 0)) atomicExch(&s_fail, 1);
    }
  } else {
    // ---------------- epilogue (warps 2-5; warp w owns TMEM lanes 32 (w & 3) ..)
    // Each 32 x 32 block of the accumulator (lane = row) goes through the
    // warp's padded shared-memory tile so that the global stores run along
    // rows (one 128- or 256-byte row segment per warp store).
    const int quarter = warp & 3;
    float* tb = epi + (warp - 2) * (32 * 33);
    // MIX: the mixing matrix as pairs (w, w), IN x OUT4, zero padded, and
    // the offset of output o = s' Dr + w_r in the second GEMM's operand
    float2* Wd = reinterpret_cast<float2*>(epi + 4 * 32 * 33);
    ll* ooff = reinterpret_cast<ll*>(Wd + 32 * 32);
    __shared__ int s_epi_ok[4];
    if constexpr (MIX) {
      const int IN = mx.Dl * mx.d2, OUT = mx.d2 * mx.Dr, OUT4 = (OUT + 3) & ~3;
      for (int e = threadIdx.x - 64; e < IN * OUT4; e += 128) {
        const int ii = e / OUT4, o = e - ii * OUT4;
        const float w = o < OUT ? (float)mx.W[ii * OUT + o] : 0.f;
        Wd[e] = make_float2(w, w);
      }
      for (int o = threadIdx.x - 64; o < OUT; o += 128) {
        const int sp = o / mx.Dr, wr = o - sp * mx.Dr;
        ooff[o] = (ll)sp * mx.ldo + (ll)wr * mx.kr;
      }
      epi_sync();
    }
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const TileIdx ti = tile_of(t, tiles_n, tiles_mn, nk_all, per_z, bmu);
      const int b = i % Cfg::NBUF, use = i / Cfg::NBUF;
      bool have = mbar_wait(&accf[b], (uint32_t)(use & 1));
      have = __all_sync(0xffffffffu, have);  // tcgen05.ld below must be warp-uniform
      if constexpr (MIX) {
        // the fused epilogue synchronises its four warps: they leave together
        if (lane == 0) s_epi_ok[quarter] = have ? 1 : 0;
        epi_sync();
        have = s_epi_ok[0] && s_epi_ok[1] && s_epi_ok[2] && s_epi_ok[3];
        epi_sync();
      }
      if (!have) {
        if (lane == 0) atomicExch(&s_fail, 1);
        break;
      }
      tc_fence_after();
      const int m0 = ti.m0, n0 = ti.nt * BN;
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * Cfg::NACC * BN);
      if constexpr (MIX) {
        // stage 32 accumulator columns of all 128 rows, then each thread
        // mixes two neighbouring (a, c) groups (c, c + 1): Dl rows x d2
        // columns of the stage each, packed FP32x2 FMAs, bf16x2 stores
        const int IN = mx.Dl * mx.d2, OUT = mx.d2 * mx.Dr, OUT4 = (OUT + 3) & ~3;
        const int ls = __ffs(mx.d2) - 1;  // d2 = 2^ls
        const int cpc2 = 16 >> ls;        // pairs of c per 32-column chunk (>= 1: d2 <= 16 here)
        const int npair = mx.apt * cpc2;
        const int et = threadIdx.x - 64, a0 = (m0 / bmu) * mx.apt;
        const bool even = (mx.kr & 1) == 0 && (mx.ldo & 1) == 0;
        float* srow = epi + (quarter * 32 + lane) * 33;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
          if (n0 + c0 >= N) break;  // uniform over the four warps
          uint32_t r[32];
          tmem_ld_32x32b_x32(lane_base + (uint32_t)c0, r);
#pragma unroll
          for (int j = 0; j < 32; ++j) srow[j] = __uint_as_float(r[j]);
          epi_sync();
          const int cb0 = (n0 + c0) >> ls;
          for (int pp = et; pp < npair; pp += 128) {
            const int al = pp / cpc2, cl = 2 * (pp - al * cpc2);
            const int a = a0 + al, c = cb0 + cl;
            if (a >= mx.chil || c >= mx.kr) continue;
            const bool two = c + 1 < mx.kr;
            float2 x[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              if (q < IN) {
                const float* e0 = epi + (al * mx.Dl + (q >> ls)) * 33 + (cl << ls) + (q & (mx.d2 - 1));
                x[q] = make_float2(e0[0], e0[mx.d2]);
              } else {
                x[q] = make_float2(0.f, 0.f);
              }
            }
            const ll base = (ll)a * mx.d2 * mx.ldo + c;
            for (int o0 = 0; o0 < OUT; o0 += 4) {
              float2 acc[4];
#pragma unroll
              for (int k = 0; k < 4; ++k) acc[k] = make_float2(0.f, 0.f);
#pragma unroll
              for (int q = 0; q < 32; ++q) {
                if (q < IN) {
                  const float4 wa = *reinterpret_cast<const float4*>(Wd + q * OUT4 + o0);
                  const float4 wb = *reinterpret_cast<const float4*>(Wd + q * OUT4 + o0 + 2);
                  acc[0] = __ffma2_rn(make_float2(wa.x, wa.y), x[q], acc[0]);
                  acc[1] = __ffma2_rn(make_float2(wa.z, wa.w), x[q], acc[1]);
                  acc[2] = __ffma2_rn(make_float2(wb.x, wb.y), x[q], acc[2]);
                  acc[3] = __ffma2_rn(make_float2(wb.z, wb.w), x[q], acc[3]);
                }
              }
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                if (o0 + k < OUT) {
                  const ll off = base + ooff[o0 + k];
                  __align__(4) __nv_bfloat16 h[2], l[2];
                  h[0] = __float2bfloat16_rn(acc[k].x);
                  h[1] = __float2bfloat16_rn(acc[k].y);
                  l[0] = __float2bfloat16_rn(acc[k].x - __bfloat162float(h[0]));  // exact differences
                  l[1] = __float2bfloat16_rn(acc[k].y - __bfloat162float(h[1]));
                  if (two && even) {
                    *reinterpret_cast<uint32_t*>(mx.hi + off) = *reinterpret_cast<const uint32_t*>(h);
                    *reinterpret_cast<uint32_t*>(mx.lo + off) = *reinterpret_cast<const uint32_t*>(l);
                  } else {
                    mx.hi[off] = h[0];
                    mx.lo[off] = l[0];
                    if (two) {
                      mx.hi[off + 1] = h[1];
                      mx.lo[off + 1] = l[1];
                    }
                  }
                }
              }
            }
          }
          epi_sync();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[b]);
        continue;
      }
      OutT* Cz = C + (ll)ti.z * M * ldc;
      const int rbase = m0 + quarter * 32;
      const int nacc = ti.nk < Cfg::NACC ? ti.nk : Cfg::NACC;  // accumulators this tile wrote
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (n0 + c0 >= N) break;  // warp-uniform
        uint32_t r[32];
        tmem_ld_32x32b_x32(lane_base + (uint32_t)c0, r);
        float acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = __uint_as_float(r[j]);
        if constexpr (Cfg::NACC > 1) {
          for (int a = 1; a < nacc; ++a) {
            tmem_ld_32x32b_x32(lane_base + (uint32_t)(a * BN + c0), r);
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = __fadd_rn(acc[j], __uint_as_float(r[j]));
          }
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) tb[lane * 33 + j] = acc[j];
        __syncwarp();
        const int col = n0 + c0 + lane;
        if (col < N) {
#pragma unroll 8
          for (int rr = 0; rr < 32; ++rr)
            if (rbase + rr < M) store_out(Cz + (ll)(rbase + rr) * ldc + col, tb[rr * 33 + lane]);
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, Cfg::TMEM_COLS);
  if (threadIdx.x == 0 && s_fail) post_status(status, SEEMPS_ERR_TIMEOUT);
}

// ----------------------------------------------------------------- host side
std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_encode{nullptr};

bool load_encode(seemps_ctx* ctx) {
  if (g_encode.load()) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    seemps_set_error(ctx, "cuTensorMapEncodeTiled unavailable");
    return false;
  }
  g_encode.store((PFN_cuTensorMapEncodeTiled_v12000)fn);  // same value from every thread
  return true;
}

seemps_status make_tmap(seemps_ctx* ctx, CUtensorMap* map, const void* base, int rows, int kp,
                        int box_rows, int box_k) {
  if (((uintptr_t)base & 15) || (kp % BK) || (box_k != 64 && box_k != 32)) {
    seemps_set_error(ctx, "tensor map: misaligned base or K not a multiple of 64");
    return SEEMPS_ERR_INVALID;
  }
  cuuint64_t gdim[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  // the swizzle spans one box row: 128 bytes (64 bf16) or 64 bytes (32 bf16)
  CUresult r = g_encode.load()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim,
                        gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        box_k == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    seemps_set_error(ctx, "cuTensorMapEncodeTiled failed (%d) rows=%d kp=%d", (int)r, rows, kp);
    return SEEMPS_ERR_CUDA;
  }
  return SEEMPS_OK;
}

template <int BN, typename OutT, int NS = 2, bool MIX = false>
seemps_status launch_tc(seemps_ctx* ctx, const SplitOperand& A, const SplitOperand& B, int Kp,
                        OutT* C, ll ldc, int ksplit = 1, const MixEpi* mix = nullptr) {
  using Cfg = TileCfg<BN, NS>;
  // set on every call (a cheap host call): correct for any device and thread
  SEEMPS_CHECK_CUDA(ctx, cudaFuncSetAttribute(tc_gemm_bf16x3_kernel<BN, OutT, NS, MIX>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              Cfg::SMEM_BYTES));
  CUtensorMap tah, tal, tal2, tbh, tbl, tbl2;
  SEEMPS_TRY(make_tmap(ctx, &tah, A.hi, A.rows, Kp, BM, Cfg::BKT));
  SEEMPS_TRY(make_tmap(ctx, &tal, A.lo, A.rows, Kp, BM, Cfg::BKT));
  SEEMPS_TRY(make_tmap(ctx, &tbh, B.hi, B.rows, Kp, BN, Cfg::BKT));
  SEEMPS_TRY(make_tmap(ctx, &tbl, B.lo, B.rows, Kp, BN, Cfg::BKT));
  if (NS == 3) {
    SEEMPS_TRY(make_tmap(ctx, &tal2, A.lo2, A.rows, Kp, BM, Cfg::BKT));
    SEEMPS_TRY(make_tmap(ctx, &tbl2, B.lo2, B.rows, Kp, BN, Cfg::BKT));
  } else {
    tal2 = tal;  // unused
    tbl2 = tbl;
  }
  // M tiles start every bmu rows: 128, or whole groups of D_l rows for the mixing
  MixEpi mx = {};
  int bmu = BM;
  if (MIX) {
    mx = *mix;
    bmu = mx.apt * mx.Dl;
    if (bmu < 1 || bmu > BM || ksplit != 1) {
      seemps_set_error(ctx, "tc_gemm: fused mixing with %d rows per tile", bmu);
      return SEEMPS_ERR_INVALID;
    }
  }
  // persistent grid: one CTA per SM (or per tile, if fewer)
  const ll tiles = (ll)ceil_div(B.rows, BN) * ceil_div(A.rows, bmu) * ksplit;
  const int nk_all = Kp / BK, per_z = ksplit > 0 ? (nk_all + ksplit - 1) / ksplit : 0;  // 64-element blocks
  if (tiles > 0x7fffffffLL || ksplit < 1 || (ll)(ksplit - 1) * per_z >= nk_all) {  // every split has K blocks
    seemps_set_error(ctx, "tc_gemm: %lld tiles (split %d) out of range", tiles, ksplit);
    return SEEMPS_ERR_INVALID;
  }
  const int grid = (int)(tiles < ctx->sm_count ? tiles : ctx->sm_count);
  PhaseTimer timer(ctx, SEEMPS_PHASE_TC_GEMM);
  tc_gemm_bf16x3_kernel<BN, OutT, NS, MIX><<<grid, 192, Cfg::SMEM_BYTES, ctx->stream>>>(
      tah, tal, tal2, tbh, tbl, tbl2, C, A.rows, B.rows, Kp, ldc, ksplit, bmu, mx, ctx->d_status, ctx->skip);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

// ----------------------------------------------------------------- split K
// With fewer 128 x 128 output tiles than SMs and a long K, the persistent
// grid would leave SMs idle: the K blocks are then shared out over ks <= 4
// CTAs per tile (each at least 16 K blocks, ks tiles x ks >= the SM count);
// each writes an FP32 partial product to the workspace and one pass adds
// them in order.  ks depends on (M, N, K) only, so both tile shapes give the
// same sums.
int split_rule(const seemps_ctx* ctx, int M, int N, int Kp) {
  const ll tiles = (ll)ceil_div(M, BM) * ceil_div(N, 128);
  const int nk = Kp / BK;
  if (tiles >= (ll)ctx->sm_count || nk < 32) return 1;
  int ks = (int)(((ll)ctx->sm_count + tiles - 1) / tiles);
  if (ks > 4) ks = 4;
  if (ks > nk / 16) ks = nk / 16;
  while (ks > 1 && ((nk + ks - 1) / ks) * (ks - 1) >= nk) --ks;  // every CTA gets K blocks
  return ks < 1 ? 1 : ks;
}

template <typename OutT>
__global__ void splitk_sum_kernel(const float* __restrict__ part, int ks, int M, int N, OutT* __restrict__ C,
                                  ll ldc, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  const ll total = (ll)M * N, stride = (ll)gridDim.x * blockDim.x;
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < total; e += stride) {
    float acc = part[e];
    for (int z = 1; z < ks; ++z) acc += part[(ll)z * total + e];
    const int m = (int)(e / N), n = (int)(e % N);
    C[(ll)m * ldc + n] = (OutT)acc;
  }
}

// The split-K GEMM: partial products in the workspace, then their sum into C.
template <int BN, typename OutT, int NS>
seemps_status launch_split(seemps_ctx* ctx, const SplitOperand& A, const SplitOperand& B, int Kp, OutT* C,
                           ll ldc, int ks, bool* done) {
  *done = false;
  WsFrame frame(ctx);
  float* part;
  const bool had_error = ctx->err[0] != 0;
  if (ws_alloc(ctx, (size_t)ks * A.rows * B.rows, &part) != SEEMPS_OK) {
    if (!had_error) ctx->err[0] = 0;  // no room: the caller runs the unsplit GEMM
    return SEEMPS_OK;
  }
  SEEMPS_TRY((launch_tc<BN, float, NS>(ctx, A, B, Kp, part, B.rows, ks)));
  splitk_sum_kernel<OutT><<<stride_grid(ctx, (ll)A.rows * B.rows, 256, 8), 256, 0, ctx->stream>>>(
      part, ks, A.rows, B.rows, C, ldc, ctx->skip);
  SEEMPS_LAUNCHED(ctx);
  *done = true;
  return SEEMPS_OK;
}

// ----------------------------------------------------------------- tile autotuner
// The 128 x 128 and 128 x 256 tile kernels form every element of C from the
// same MMAs in the same order (their results are bit-identical); which one
// is faster depends on the shape (waves over the SMs, the epilogue's share).
// seemps_autotune times both on the GEMMs of a pair update at given sizes and
// records the winner per (device, M, N, Kp, output type) in a process-wide
// table; a context with autotuning on takes the recorded winner, and the
// SM-count rule below for shapes never tuned.
using TuneKey = std::tuple<int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

int tune_lookup(const TuneKey& k) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(k);
  return it == g_tune.end() ? 0 : it->second;
}

int tile_rule(const seemps_ctx* ctx, int M, int N) {
  // fewer than ~1.5 waves of 128x256 tiles: use 128x128 tiles for occupancy
  const ll tiles256 = (ll)ceil_div(M, BM) * ceil_div(N, 256);
  return (N > 128 && tiles256 >= (ll)ctx->sm_count * 3 / 2) ? 256 : 128;
}

template <typename OutT>
seemps_status tc_gemm_any(seemps_ctx* ctx, const SplitOperand& A, const SplitOperand& B, int Kp,
                          OutT* C, ll ldc) {
  if (A.rows <= 0 || B.rows <= 0) return SEEMPS_OK;
  if (!tc_available(ctx)) {
    seemps_set_error(ctx, "bf16x3 tensor-core path needs an sm_103 (GB300) device, found sm_%d%d",
                     ctx->cc_major, ctx->cc_minor);
    return SEEMPS_ERR_UNSUPPORTED;
  }
  if (!load_encode(ctx)) return SEEMPS_ERR_UNSUPPORTED;
  if (Kp <= 0 || Kp % BK) {
    seemps_set_error(ctx, "tc_gemm: Kp=%d not a positive multiple of 64", Kp);
    return SEEMPS_ERR_INVALID;
  }
  const int ks = split_rule(ctx, A.rows, B.rows, Kp);
  bool done = false;
  if (A.lo2 || B.lo2) {
    if (!A.lo2 || !B.lo2) {
      seemps_set_error(ctx, "tc_gemm: both operands need a third plane for the six-product GEMM");
      return SEEMPS_ERR_INVALID;
    }
    if (ks > 1) SEEMPS_TRY((launch_split<128, OutT, 3>(ctx, A, B, Kp, C, ldc, ks, &done)));
    if (done) return SEEMPS_OK;
    return launch_tc<128, OutT, 3>(ctx, A, B, Kp, C, ldc);
  }
  int bn = tile_rule(ctx, A.rows, B.rows);
  if (ctx->autotune) {
    const int t = tune_lookup(TuneKey(ctx->device, A.rows, B.rows, Kp, (int)sizeof(OutT)));
    if (t) {
      bn = t;
      ctx->tune_hits++;
    }
  }
  if (ks > 1) {
    if (bn == 256) SEEMPS_TRY((launch_split<256, OutT, 2>(ctx, A, B, Kp, C, ldc, ks, &done)));
    else SEEMPS_TRY((launch_split<128, OutT, 2>(ctx, A, B, Kp, C, ldc, ks, &done)));
    if (done) return SEEMPS_OK;
  }
  if (bn == 256) return launch_tc<256, OutT>(ctx, A, B, Kp, C, ldc);
  return launch_tc<128, OutT>(ctx, A, B, Kp, C, ldc);
}

// Times both tile kernels on an M x N x Kp GEMM (operands from the workspace,
// filled with a constant) and records the faster.  Synchronises the stream;
// not for use under stream capture.  A shape whose operands do not fit in the
// workspace is left untuned (the rule applies).
template <typename OutT>
seemps_status tune_shape(seemps_ctx* ctx, int M, int N, int Kp, int* tuned) {
  if (M <= 0 || N <= 0 || Kp <= 0) return SEEMPS_OK;
  const TuneKey key(ctx->device, M, N, Kp, (int)sizeof(OutT));
  if (tune_lookup(key)) return SEEMPS_OK;
  WsFrame frame(ctx);
  __nv_bfloat16 *ah, *al, *bh, *bl;
  OutT* C;
  const bool had_error = ctx->err[0] != 0;
  if (ws_alloc(ctx, (size_t)M * Kp, &ah) != SEEMPS_OK || ws_alloc(ctx, (size_t)M * Kp, &al) != SEEMPS_OK ||
      ws_alloc(ctx, (size_t)N * Kp, &bh) != SEEMPS_OK || ws_alloc(ctx, (size_t)N * Kp, &bl) != SEEMPS_OK ||
      ws_alloc(ctx, (size_t)M * N, &C) != SEEMPS_OK) {
    if (!had_error) ctx->err[0] = 0;  // not an error: the shape stays on the rule
    return SEEMPS_OK;
  }
  // bf16 0x3c3c (about 0.0115) everywhere: finite, nonzero operands
  SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(ah, 0x3c, (size_t)M * Kp * 2, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(al, 0x3c, (size_t)M * Kp * 2, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(bh, 0x3c, (size_t)N * Kp * 2, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(bl, 0x3c, (size_t)N * Kp * 2, ctx->stream));
  const SplitOperand A = {ah, al, M, nullptr}, B = {bh, bl, N, nullptr};
  const int* saved_skip = ctx->skip;
  const int saved_timing = ctx->timing;
  ctx->skip = nullptr;
  ctx->timing = 0;
  cudaEvent_t ev[5];
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) e = nullptr;
  seemps_status rc = SEEMPS_OK;
  float best[2] = {1e30f, 1e30f};
  // the path the GEMM takes in use: split K when the rule splits it
  const int ks = split_rule(ctx, M, N, Kp);
  auto run = [&](int bn) -> seemps_status {
    if (ks > 1) {
      bool done = false;
      seemps_status r = bn == 256 ? launch_split<256, OutT, 2>(ctx, A, B, Kp, C, N, ks, &done)
                                  : launch_split<128, OutT, 2>(ctx, A, B, Kp, C, N, ks, &done);
      if (r != SEEMPS_OK || done) return r;
    }
    return bn == 256 ? launch_tc<256, OutT>(ctx, A, B, Kp, C, N) : launch_tc<128, OutT>(ctx, A, B, Kp, C, N);
  };
  if (ev[0] && ev[1] && ev[2] && ev[3] && ev[4]) {
    // one untimed launch of each, then two timed rounds, alternating
    rc = run(128);
    if (rc == SEEMPS_OK) rc = run(256);
    for (int round = 0; round < 2 && rc == SEEMPS_OK; ++round) {
      cudaEventRecord(ev[0], ctx->stream);
      rc = run(128);
      cudaEventRecord(ev[1], ctx->stream);
      if (rc == SEEMPS_OK) rc = run(256);
      cudaEventRecord(ev[2], ctx->stream);
      if (rc != SEEMPS_OK) break;
      if (cudaEventSynchronize(ev[2]) != cudaSuccess) {
        seemps_set_error(ctx, "autotune: event synchronisation failed");
        rc = SEEMPS_ERR_CUDA;
        break;
      }
      float t128 = 0.f, t256 = 0.f;
      cudaEventElapsedTime(&t128, ev[0], ev[1]);
      cudaEventElapsedTime(&t256, ev[1], ev[2]);
      best[0] = t128 < best[0] ? t128 : best[0];
      best[1] = t256 < best[1] ? t256 : best[1];
    }
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  ctx->skip = saved_skip;
  ctx->timing = saved_timing;
  SEEMPS_TRY(rc);
  if (best[0] < 1e30f) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = best[1] < best[0] ? 256 : 128;
    ctx->tune_shapes++;
    if (tuned) ++*tuned;
  }
  return SEEMPS_OK;
}

// ----------------------------------------------------------------- split kernels
// a = hi + lo + O(2^-16 |a|); the input is FP64 or FP32 (the FP32 Krylov
// basis of the mixed sweep).
template <typename TI>
__device__ __forceinline__ void split_one(TI a, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  __nv_bfloat16 h = __float2bfloat16_rn((float)a);
  TI rem = a - (TI)__bfloat162float(h);
  *hi = h;
  *lo = __float2bfloat16_rn((float)rem);
}

// a = hi + lo + lo2 + O(2^-24 |a|): each remainder formed in the input's
// precision before its bf16 rounding
template <typename TI>
__device__ __forceinline__ void split_one(TI a, __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2) {
  const __nv_bfloat16 h = __float2bfloat16_rn((float)a);
  const TI r1 = a - (TI)__bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn((float)r1);
  const TI r2 = r1 - (TI)__bfloat162float(m);
  *hi = h;
  *lo = m;
  *lo2 = __float2bfloat16_rn((float)r2);
}

// out[r][c] for c < Cp; zero for c >= C.
template <typename TI>
__global__ void split_rows_kernel(const TI* __restrict__ in, ll ld, int R, int C, int Cp,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                  __nv_bfloat16* __restrict__ lo2, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  const ll total = (ll)R * Cp;
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < total; i += (ll)gridDim.x * blockDim.x) {
    const int r = (int)(i / Cp), c = (int)(i % Cp);
    TI a = (c < C) ? in[(ll)r * ld + c] : TI(0);
    if (lo2) split_one(a, hi + i, lo + i, lo2 + i);
    else split_one(a, hi + i, lo + i);
  }
}

// out[c'][r] = in[r][c] for r < Rp (zero for r >= R), 64 x 64 tiles through
// shared memory so that both the read (along c) and the write (pairs of r,
// 4-byte bf16x2 stores) are coalesced; c' = c, or with pk > 0 (C = q pk) the
// column c = s pk + j goes to row j q + s.  Rp is a multiple of 64.
template <typename TI>
__global__ void __launch_bounds__(256) split_transpose_kernel(const TI* __restrict__ in, ll ld, int R, int C,
                                                              int Rp, __nv_bfloat16* __restrict__ hi,
                                                              __nv_bfloat16* __restrict__ lo,
                                                              __nv_bfloat16* __restrict__ lo2, int pk,
                                                              const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  __shared__ TI tile[64][65];
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  {
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
    for (int j = ty; j < 64; j += 4) {
      const int r = r0 + j, c = c0 + tx;
      tile[j][tx] = (r < R && c < C) ? in[(ll)r * ld + c] : TI(0);
    }
  }
  __syncthreads();
  const int pr = threadIdx.x & 31, cy = threadIdx.x >> 5;  // 32 row pairs x 8 columns
  for (int j = cy; j < 64; j += 8) {
    const int c = c0 + j, r = r0 + 2 * pr;
    if (c < C && r < Rp) {
      const int cr = pk > 0 ? (c % pk) * (C / pk) + c / pk : c;
      const ll o = (ll)cr * Rp + r;
      __align__(4) __nv_bfloat16 h[2], l[2], m[2];
      if (lo2) {
        split_one(tile[2 * pr][j], &h[0], &l[0], &m[0]);
        split_one(tile[2 * pr + 1][j], &h[1], &l[1], &m[1]);
        *reinterpret_cast<uint32_t*>(lo2 + o) = *reinterpret_cast<const uint32_t*>(m);
      } else {
        split_one(tile[2 * pr][j], &h[0], &l[0]);
        split_one(tile[2 * pr + 1][j], &h[1], &l[1]);
      }
      *reinterpret_cast<uint32_t*>(hi + o) = *reinterpret_cast<const uint32_t*>(h);
      *reinterpret_cast<uint32_t*>(lo + o) = *reinterpret_cast<const uint32_t*>(l);
    }
  }
}

template <typename TI>
seemps_status split_any(seemps_ctx* ctx, const TI* in, ll ld, int R, int C, bool transpose,
                        __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2 = nullptr, int pk = 0) {
  if (R <= 0 || C <= 0) return SEEMPS_OK;
  if (!transpose) {
    const int Cp = (int)round_up(C, BK);
    split_rows_kernel<TI><<<stride_grid(ctx, (ll)R * Cp, 256, 8), 256, 0, ctx->stream>>>(in, ld, R, C, Cp, hi,
                                                                                          lo, lo2, ctx->skip);
  } else {
    const int Rp = (int)round_up(R, BK);
    dim3 grid(ceil_div(C, 64), Rp / 64);
    if (grid.y > 65535) {
      seemps_set_error(ctx, "split_transpose: too many rows");
      return SEEMPS_ERR_INVALID;
    }
    split_transpose_kernel<TI><<<grid, 256, 0, ctx->stream>>>(in, ld, R, C, Rp, hi, lo, lo2, pk, ctx->skip);
  }
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

}  // namespace

bool tc_available(seemps_ctx* ctx) { return ctx->cc_major == 10 && ctx->cc_minor == 3; }

// The two-product-plane bf16x3 GEMMs of one pair update at the given sizes:
// the effective operator's two GEMMs (FP32 output for the Krylov basis, FP64
// for the other callers), the two-site tensor and the split's second factor.
extern "C" seemps_status seemps_autotune(seemps_ctx* ctx, const seemps_pair_dims* dm, int* tuned_out) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, dm, "autotune: null dims");
  SEEMPS_REQUIRE(ctx, dm->chi_l > 0 && dm->chi_r > 0 && dm->d > 0 && dm->D_l > 0 && dm->D_m > 0 && dm->D_r > 0,
                 "autotune: non-positive dimension");
  SEEMPS_REQUIRE(ctx, tc_available(ctx), "autotune: the tensor-core path needs an sm_103 device");
  if (!load_encode(ctx)) return SEEMPS_ERR_UNSUPPORTED;
  int tuned = 0;
  const int cl = dm->chi_l, cr = dm->chi_r, d = dm->d, d2 = d * d;
  const int Dl = dm->D_l, Dr = dm->D_r, Dm = dm->D_m;
  auto kp = [](ll k) { return (int)round_up(k, BK); };
  // effective operator: T1 = L theta, y = T2 R
  SEEMPS_TRY(tune_shape<float>(ctx, cl * Dl, d2 * cr, kp(cl), &tuned));
  SEEMPS_TRY(tune_shape<float>(ctx, cl * d2, cr, kp((ll)Dr * cr), &tuned));
  SEEMPS_TRY(tune_shape<double>(ctx, cl * d2, cr, kp((ll)Dr * cr), &tuned));
  // (the environment updates run the six-product GEMM on 128-wide tiles and
  // have no tile choice.)  The new bond chi_m: at most min(chi_l d, d chi_r),
  // and in the bulk of a sweep at chi_max the larger of the two outer bonds.
  (void)Dm;
  int cm = dm->chi_l * d < d * dm->chi_r ? dm->chi_l * d : d * dm->chi_r;
  const int cmax = cl > cr ? cl : cr;
  if (cmax < cm) cm = cmax;
  // two-site tensor and the split's second factor
  SEEMPS_TRY(tune_shape<double>(ctx, cl * d, d * cr, kp(cm), &tuned));
  SEEMPS_TRY(tune_shape<double>(ctx, cm, d * cr, kp((ll)cl * d), &tuned));
  SEEMPS_TRY(tune_shape<double>(ctx, cl * d, cm, kp((ll)d * cr), &tuned));
  SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (tuned_out) *tuned_out = tuned;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_set_autotune(seemps_ctx* ctx, int enabled) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  ctx->autotune = enabled ? 1 : 0;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_autotune_stats(const seemps_ctx* ctx, long long* hits_out, long long* shapes_out,
                                               int* table_size_out) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  if (hits_out) *hits_out = ctx->tune_hits;
  if (shapes_out) *shapes_out = ctx->tune_shapes;
  if (table_size_out) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    *table_size_out = (int)g_tune.size();
  }
  return SEEMPS_OK;
}

seemps_status tc_gemm_f32out(seemps_ctx* ctx, const SplitOperand& A, const SplitOperand& B, int Kp,
                             float* C, ll ldc) {
  return tc_gemm_any<float>(ctx, A, B, Kp, C, ldc);
}

seemps_status tc_gemm_f64out(seemps_ctx* ctx, const SplitOperand& A, const SplitOperand& B, int Kp,
                             double* C, ll ldc) {
  return tc_gemm_any<double>(ctx, A, B, Kp, C, ldc);
}

bool mix_epi_ok(int Dl, int d2, int Dr) {
  if (d2 < 1 || d2 > 16 || (d2 & (d2 - 1)) || Dl < 1 || Dr < 1 || Dl * d2 > 32 || d2 * Dr > 32) return false;
  const int apt = BM / Dl;
  return 8 * (BM - apt * Dl) <= BM;
}

seemps_status tc_gemm_mix(seemps_ctx* ctx, const SplitOperand& A, const SplitOperand& B, int Kp,
                          const MixEpi& mx) {
  if (A.rows <= 0 || B.rows <= 0) return SEEMPS_OK;
  if (!tc_available(ctx)) {
    seemps_set_error(ctx, "bf16x3 tensor-core path needs an sm_103 (GB300) device, found sm_%d%d",
                     ctx->cc_major, ctx->cc_minor);
    return SEEMPS_ERR_UNSUPPORTED;
  }
  if (!load_encode(ctx)) return SEEMPS_ERR_UNSUPPORTED;
  if (Kp <= 0 || Kp % BK || !mix_epi_ok(mx.Dl, mx.d2, mx.Dr) || mx.apt != BM / mx.Dl ||
      A.rows != mx.chil * mx.Dl || B.rows != mx.d2 * mx.kr) {
    seemps_set_error(ctx, "tc_gemm_mix: unsupported shape");
    return SEEMPS_ERR_INVALID;
  }
  // the tile of the plain GEMM of the same shape (rule, or the autotuner's winner)
  int bn = tile_rule(ctx, A.rows, B.rows);
  if (ctx->autotune) {
    const int t = tune_lookup(TuneKey(ctx->device, A.rows, B.rows, Kp, (int)sizeof(float)));
    if (t) {
      bn = t;
      ctx->tune_hits++;
    }
  }
  if (bn == 256) return launch_tc<256, float, 2, true>(ctx, A, B, Kp, nullptr, 0, 1, &mx);
  return launch_tc<128, float, 2, true>(ctx, A, B, Kp, nullptr, 0, 1, &mx);
}

seemps_status split_bf16_perm(seemps_ctx* ctx, const double* in, ll ld, int R, int C, int kr,
                              __nv_bfloat16* hi, __nv_bfloat16* lo) {
  return split_any<double>(ctx, in, ld, R, C, true, hi, lo, nullptr, kr);
}

seemps_status split_bf16_perm(seemps_ctx* ctx, const float* in, ll ld, int R, int C, int kr,
                              __nv_bfloat16* hi, __nv_bfloat16* lo) {
  return split_any<float>(ctx, in, ld, R, C, true, hi, lo, nullptr, kr);
}

seemps_status split_bf16(seemps_ctx* ctx, const double* in, ll ld, int R, int C, bool transpose,
                         __nv_bfloat16* hi, __nv_bfloat16* lo) {
  return split_any<double>(ctx, in, ld, R, C, transpose, hi, lo);
}

seemps_status split_bf16(seemps_ctx* ctx, const float* in, ll ld, int R, int C, bool transpose,
                         __nv_bfloat16* hi, __nv_bfloat16* lo) {
  return split_any<float>(ctx, in, ld, R, C, transpose, hi, lo);
}

seemps_status split_bf16_3(seemps_ctx* ctx, const double* in, ll ld, int R, int C, bool transpose,
                           __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2) {
  return split_any<double>(ctx, in, ld, R, C, transpose, hi, lo, lo2);
}
