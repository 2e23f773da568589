// Contractions of the sweep: the quadratic- and antilinear-form environment
// updates and the effective operator of the active pair (Sect. 2.5), in FP64
// (CUDA-core GEMM) or split bf16x3 (tcgen05 GEMM).
//
// Every contraction is two large GEMMs around a small "mix" with the MPO
// tensor(s).  The mix kernel is generic: for each (outer, inner) index pair
// it maps IN input values to OUT output values through a dense IN x OUT
// matrix built from the MPO, with reads and writes coalesced along `inner`
// (inputs in registers for IN <= 32, otherwise staged 32 inner indices per
// block in shared memory).
#include <type_traits>

#include "contract.cuh"
#include "timing.cuh"

namespace {

template <typename TIn, typename TW, bool SPLIT>
__global__ void __launch_bounds__(256) mix_kernel(MixArgs a, const TIn* __restrict__ in,
                                                  const double* __restrict__ Wmat,
                                                  double* __restrict__ out64,
                                                  __nv_bfloat16* __restrict__ hi,
                                                  __nv_bfloat16* __restrict__ lo,
                                                  __nv_bfloat16* __restrict__ lo2,
                                                  const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  extern __shared__ __align__(16) unsigned char mix_smem[];
  TW* Ws = reinterpret_cast<TW*>(mix_smem);                       // [IN][OUT]
  TIn* slab = reinterpret_cast<TIn*>(mix_smem + (((size_t)a.IN * a.OUT * sizeof(TW) + 15) & ~(size_t)15));  // [IN][32]
  const int outer = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int inner = blockIdx.x * 32 + lane;
  const bool live = inner < a.n_inner;
  for (int e = threadIdx.x; e < a.IN * a.OUT; e += blockDim.x) Ws[e] = (TW)Wmat[e];
  const TIn* ib = in + (ll)outer * a.in_so;
  for (int i = warp; i < a.IN; i += nwarp) {
    ll off = (ll)(i / a.in_n2) * a.in_s1 + (ll)(i % a.in_n2) * a.in_s2 + inner;
    slab[i * 32 + lane] = live ? ib[off] : (TIn)0;
  }
  __syncthreads();
  if (!live) return;
  for (int o = warp; o < a.OUT; o += nwarp) {
    TW acc = 0;
    for (int i = 0; i < a.IN; ++i) acc += Ws[i * a.OUT + o] * (TW)slab[i * 32 + lane];
    ll off = (ll)outer * a.out_so + (ll)(o / a.out_m2) * a.out_t1 + (ll)(o % a.out_m2) * a.out_t2 +
             (ll)inner * a.out_ti;
    if (SPLIT) {
      __nv_bfloat16 h = __float2bfloat16_rn((float)acc);
      hi[off] = h;
      const TW r = acc - (TW)__bfloat162float(h);  // exact in TW
      if (lo2) {
        const __nv_bfloat16 m = __float2bfloat16_rn((float)r);
        lo[off] = m;
        lo2[off] = __float2bfloat16_rn((float)(r - (TW)__bfloat162float(m)));
      } else {
        lo[off] = __float2bfloat16_rn((float)r);
      }
    } else {
      out64[off] = (double)acc;
    }
  }
}

// Register variant for IN <= MIX_MAXIN: one thread per (outer, inner) pair
// keeps its IN inputs in registers and forms all OUT outputs; loads and
// stores are coalesced along `inner`, the mixing matrix and the offsets of
// the IN rows / OUT rows are broadcast from shared memory.
constexpr int MIX_MAXIN = 32;
constexpr int MIX_NT = 256;
template <typename TIn, typename TW, bool SPLIT>
__global__ void __launch_bounds__(MIX_NT) mix_reg_kernel(MixArgs a, const TIn* __restrict__ in,
                                                         const double* __restrict__ Wmat,
                                                         double* __restrict__ out64,
                                                         __nv_bfloat16* __restrict__ hi,
                                                         __nv_bfloat16* __restrict__ lo,
                                                         __nv_bfloat16* __restrict__ lo2, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  extern __shared__ __align__(16) unsigned char mix_smem[];
  TW* Ws = reinterpret_cast<TW*>(mix_smem);  // [IN][OUT]
  ll* ioff = reinterpret_cast<ll*>(mix_smem + (((size_t)a.IN * a.OUT * sizeof(TW) + 15) & ~(size_t)15));
  ll* ooff = ioff + a.IN;
  for (int e = threadIdx.x; e < a.IN * a.OUT; e += MIX_NT) Ws[e] = (TW)Wmat[e];
  for (int i = threadIdx.x; i < a.IN; i += MIX_NT)
    ioff[i] = (ll)(i / a.in_n2) * a.in_s1 + (ll)(i % a.in_n2) * a.in_s2;
  for (int o = threadIdx.x; o < a.OUT; o += MIX_NT)
    ooff[o] = (ll)(o / a.out_m2) * a.out_t1 + (ll)(o % a.out_m2) * a.out_t2;
  __syncthreads();
  const int inner = blockIdx.x * MIX_NT + threadIdx.x;
  if (inner >= a.n_inner) return;
  const int outer = blockIdx.y;
  const TIn* ib = in + (ll)outer * a.in_so + inner;
  TW x[MIX_MAXIN];
#pragma unroll
  for (int i = 0; i < MIX_MAXIN; ++i) x[i] = i < a.IN ? (TW)ib[ioff[i]] : TW(0);
  const ll ob = (ll)outer * a.out_so + (ll)inner * a.out_ti;
  for (int o = 0; o < a.OUT; ++o) {
    TW acc = 0;
#pragma unroll
    for (int i = 0; i < MIX_MAXIN; ++i)
      if (i < a.IN) acc += Ws[i * a.OUT + o] * x[i];
    const ll off = ob + ooff[o];
    if (SPLIT) {
      const __nv_bfloat16 h = __float2bfloat16_rn((float)acc);
      hi[off] = h;
      const TW r = acc - (TW)__bfloat162float(h);  // exact in TW
      if (lo2) {
        const __nv_bfloat16 m = __float2bfloat16_rn((float)r);
        lo[off] = m;
        lo2[off] = __float2bfloat16_rn((float)(r - (TW)__bfloat162float(m)));
      } else {
        lo[off] = __float2bfloat16_rn((float)r);
      }
    } else {
      out64[off] = (double)acc;
    }
  }
}

// Vector variant for the bf16x3 path (FP32 input, bf16 hi/lo output): a
// thread forms all OUT outputs of 2 consecutive inner elements, so that each
// 8-byte input load and two 16-byte broadcasts of four mixing coefficients
// (stored as pairs (w, w)) feed 4 packed FP32x2 FMAs, bit-identical to 8
// scalar ones (the scalar kernel spends a shared-memory load and index
// arithmetic per FMA and is instruction-bound; two elements per thread
// rather than four halve the input registers, so more warps cover the loads).  Resident blocks walk the
// (outer, inner block) items, loading the matrix once.  Needs the inner index
// contiguous on both sides, n_inner and every row offset a multiple of 4,
// and IN <= NI.
template <int NI>
__global__ void __launch_bounds__(MIX_NT) mix_vec_kernel(MixArgs a, const float* __restrict__ in,
                                                         const double* __restrict__ Wmat,
                                                         __nv_bfloat16* __restrict__ hi,
                                                         __nv_bfloat16* __restrict__ lo,
                                                         __nv_bfloat16* __restrict__ lo2, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  extern __shared__ __align__(16) unsigned char mix_smem[];
  const int OUT4 = (a.OUT + 3) & ~3;
  // [IN][OUT4] pairs (w, w), zero padded: one packed FMA applies w to two inner elements
  float2* Wd = reinterpret_cast<float2*>(mix_smem);
  ll* ioff = reinterpret_cast<ll*>(mix_smem + (((size_t)a.IN * OUT4 * sizeof(float2) + 15) & ~(size_t)15));
  ll* ooff = ioff + a.IN;
  for (int e = threadIdx.x; e < a.IN * OUT4; e += MIX_NT) {
    const int i = e / OUT4, o = e % OUT4;
    const float w = o < a.OUT ? (float)Wmat[i * a.OUT + o] : 0.f;
    Wd[e] = make_float2(w, w);
  }
  for (int i = threadIdx.x; i < a.IN; i += MIX_NT)
    ioff[i] = (ll)(i / a.in_n2) * a.in_s1 + (ll)(i % a.in_n2) * a.in_s2;
  for (int o = threadIdx.x; o < a.OUT; o += MIX_NT)
    ooff[o] = (ll)(o / a.out_m2) * a.out_t1 + (ll)(o % a.out_m2) * a.out_t2;
  __syncthreads();
  // grid-stride over (outer, block of MIX_NT x 2 inner elements): the
  // matrix and offsets above are loaded once per resident block
  const int nx = (int)((a.n_inner / 2 + MIX_NT - 1) / MIX_NT);
  const ll items = (ll)a.n_outer * nx;
  for (ll item = blockIdx.x; item < items; item += gridDim.x) {
    const int outer = (int)(item / nx);
    const ll c2 = 2 * ((item - (ll)outer * nx) * MIX_NT + threadIdx.x);
    if (c2 >= a.n_inner) continue;
    const float* ib = in + (ll)outer * a.in_so + c2;
    float2 x[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i)
      x[i] = i < a.IN ? *reinterpret_cast<const float2*>(ib + ioff[i]) : make_float2(0.f, 0.f);
    const ll ob = (ll)outer * a.out_so + c2;
    for (int o0 = 0; o0 < a.OUT; o0 += 4) {
      float2 acc[4];  // output o0 + k, inner elements (0, 1)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        if (i < a.IN) {
          const float4 wa = *reinterpret_cast<const float4*>(Wd + i * OUT4 + o0);
          const float4 wb = *reinterpret_cast<const float4*>(Wd + i * OUT4 + o0 + 2);
          acc[0] = __ffma2_rn(make_float2(wa.x, wa.y), x[i], acc[0]);
          acc[1] = __ffma2_rn(make_float2(wa.z, wa.w), x[i], acc[1]);
          acc[2] = __ffma2_rn(make_float2(wb.x, wb.y), x[i], acc[2]);
          acc[3] = __ffma2_rn(make_float2(wb.z, wb.w), x[i], acc[3]);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (o0 + k < a.OUT) {
          __align__(4) __nv_bfloat16 h[2], l[2], l2[2];
          const float v[2] = {acc[k].x, acc[k].y};
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            h[e] = __float2bfloat16_rn(v[e]);
            const float r = v[e] - __bfloat162float(h[e]);  // exact in FP32
            l[e] = __float2bfloat16_rn(r);
            l2[e] = __float2bfloat16_rn(r - __bfloat162float(l[e]));
          }
          const ll off = ob + ooff[o0 + k];
          *reinterpret_cast<uint32_t*>(hi + off) = *reinterpret_cast<const uint32_t*>(h);
          *reinterpret_cast<uint32_t*>(lo + off) = *reinterpret_cast<const uint32_t*>(l);
          if (lo2) *reinterpret_cast<uint32_t*>(lo2 + off) = *reinterpret_cast<const uint32_t*>(l2);
        }
      }
    }
  }
}

// Wide MPO blocks in the bf16x3 path (IN above the register-input kernel's
// 32, OUT <= NO): one thread per (outer, inner) pair keeps all OUT
// accumulators in registers and streams its IN inputs once (loads coalesced
// along `inner`); each input meets four mixing coefficients per 16-byte
// broadcast load of the zero-padded matrix in shared memory.
constexpr int MIX_ACC_NT = 128;
template <int NO>
__global__ void __launch_bounds__(MIX_ACC_NT) mix_acc_kernel(MixArgs a, const float* __restrict__ in,
                                                             const double* __restrict__ Wmat,
                                                             __nv_bfloat16* __restrict__ hi,
                                                             __nv_bfloat16* __restrict__ lo,
                                                             __nv_bfloat16* __restrict__ lo2, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  extern __shared__ __align__(16) unsigned char mix_smem[];
  float* Ws = reinterpret_cast<float*>(mix_smem);  // [IN][NO], zero padded
  ll* ioff = reinterpret_cast<ll*>(mix_smem + (size_t)a.IN * NO * sizeof(float));
  ll* ooff = ioff + a.IN;
  for (int e = threadIdx.x; e < a.IN * NO; e += MIX_ACC_NT) {
    const int i = e / NO, o = e % NO;
    Ws[e] = o < a.OUT ? (float)Wmat[i * a.OUT + o] : 0.f;
  }
  for (int i = threadIdx.x; i < a.IN; i += MIX_ACC_NT)
    ioff[i] = (ll)(i / a.in_n2) * a.in_s1 + (ll)(i % a.in_n2) * a.in_s2;
  for (int o = threadIdx.x; o < a.OUT; o += MIX_ACC_NT)
    ooff[o] = (ll)(o / a.out_m2) * a.out_t1 + (ll)(o % a.out_m2) * a.out_t2;
  __syncthreads();
  const int inner = blockIdx.x * MIX_ACC_NT + threadIdx.x;
  if (inner >= a.n_inner) return;
  const float* ib = in + (ll)blockIdx.y * a.in_so + inner;
  float acc[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) acc[o] = 0.f;
  for (int i = 0; i < a.IN; ++i) {
    const float x = ib[ioff[i]];
    const float4* w4 = reinterpret_cast<const float4*>(Ws + (size_t)i * NO);
#pragma unroll
    for (int q = 0; q < NO / 4; ++q) {
      const float4 w = w4[q];
      acc[4 * q] = fmaf(w.x, x, acc[4 * q]);
      acc[4 * q + 1] = fmaf(w.y, x, acc[4 * q + 1]);
      acc[4 * q + 2] = fmaf(w.z, x, acc[4 * q + 2]);
      acc[4 * q + 3] = fmaf(w.w, x, acc[4 * q + 3]);
    }
  }
  const ll ob = (ll)blockIdx.y * a.out_so + (ll)inner * a.out_ti;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    if (o < a.OUT) {
      const ll off = ob + ooff[o];
      const __nv_bfloat16 h = __float2bfloat16_rn(acc[o]);
      const float r = acc[o] - __bfloat162float(h);  // exact in FP32
      hi[off] = h;
      if (lo2) {
        const __nv_bfloat16 m = __float2bfloat16_rn(r);
        lo[off] = m;
        lo2[off] = __float2bfloat16_rn(r - __bfloat162float(m));
      } else {
        lo[off] = __float2bfloat16_rn(r);
      }
    }
  }
}

template <int NO>
seemps_status launch_mix_acc(seemps_ctx* ctx, const MixArgs& a, const float* in, const double* Wmat,
                             __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2) {
  const size_t smem = (size_t)a.IN * NO * sizeof(float) + (size_t)(a.IN + a.OUT) * sizeof(ll);
  // one fixed limit per kernel: several host threads (sweep_batch) launch it concurrently
  if (smem > 220 * 1024) {
    seemps_set_error(ctx, "mix: %zu bytes of mixing matrix exceed shared memory", smem);
    return SEEMPS_ERR_INVALID;
  }
  if (smem > 48 * 1024)
    SEEMPS_CHECK_CUDA(ctx, cudaFuncSetAttribute(mix_acc_kernel<NO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                220 * 1024));
  dim3 grid(ceil_div(a.n_inner, MIX_ACC_NT), a.n_outer);
  mix_acc_kernel<NO><<<grid, MIX_ACC_NT, smem, ctx->stream>>>(a, in, Wmat, hi, lo, lo2, ctx->skip);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

// The vector kernel applies: FP32 input, split output, inner contiguous,
// every offset a multiple of 4 elements, 16-byte (input) / 8-byte (output)
// aligned bases.
static bool mix_vec_ok(const MixArgs& a, const void* in, const void* hi, const void* lo, const void* lo2) {
  if (a.out_ti != 1 || a.IN > 32 || (a.n_inner & 3) || (a.in_so & 3) || (a.out_so & 3)) return false;
  if (((uintptr_t)in & 15) || ((uintptr_t)hi & 7) || ((uintptr_t)lo & 7) || ((uintptr_t)lo2 & 7)) return false;
  for (int i = 0; i < a.IN; ++i)
    if ((((ll)(i / a.in_n2) * a.in_s1 + (ll)(i % a.in_n2) * a.in_s2) & 3)) return false;
  for (int o = 0; o < a.OUT; ++o)
    if ((((ll)(o / a.out_m2) * a.out_t1 + (ll)(o % a.out_m2) * a.out_t2) & 3)) return false;
  return true;
}

template <int NI>
seemps_status launch_mix_vec(seemps_ctx* ctx, const MixArgs& a, const float* in, const double* Wmat,
                             __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2) {
  const int OUT4 = (a.OUT + 3) & ~3;
  const size_t smem = (((size_t)a.IN * OUT4 * sizeof(float2) + 15) & ~(size_t)15) +
                      (size_t)(a.IN + a.OUT) * sizeof(ll);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mix_vec_kernel<NI>, MIX_NT, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const ll items = (ll)a.n_outer * ceil_div(a.n_inner / 2, MIX_NT);
  const ll cap = (ll)per_sm * ctx->sm_count;
  const int grid = (int)(items < cap ? (items > 0 ? items : 1) : cap);
  mix_vec_kernel<NI><<<grid, MIX_NT, smem, ctx->stream>>>(a, in, Wmat, hi, lo, lo2, ctx->skip);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

template <typename TIn, typename TW, bool SPLIT>
seemps_status launch_mix(seemps_ctx* ctx, const MixArgs& a, const TIn* in, const double* Wmat,
                         double* out64, __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2 = nullptr) {
  if (a.n_outer <= 0 || a.n_inner <= 0) return SEEMPS_OK;
  if constexpr (SPLIT && std::is_same<TIn, float>::value) {
    if (a.n_outer <= 65535 && mix_vec_ok(a, in, hi, lo, lo2)) {
      if (a.IN <= 12) return launch_mix_vec<12>(ctx, a, in, Wmat, hi, lo, lo2);
      if (a.IN <= 20) return launch_mix_vec<20>(ctx, a, in, Wmat, hi, lo, lo2);
      return launch_mix_vec<32>(ctx, a, in, Wmat, hi, lo, lo2);
    }
  }
  if constexpr (SPLIT && std::is_same<TIn, float>::value) {
    // wide MPO blocks: accumulators in registers (up to 128 outputs, <= 200 KB of coefficients)
    if (a.IN > MIX_MAXIN && a.n_outer <= 65535 && (size_t)a.IN * 128 * 4 <= 200 * 1024) {
      if (a.OUT <= 64) return launch_mix_acc<64>(ctx, a, in, Wmat, hi, lo, lo2);
      if (a.OUT <= 128) return launch_mix_acc<128>(ctx, a, in, Wmat, hi, lo, lo2);
    }
  }
  if (a.IN <= MIX_MAXIN && a.n_outer <= 65535) {
    const size_t smem = (((size_t)a.IN * a.OUT * sizeof(TW) + 15) & ~(size_t)15) +
                        (size_t)(a.IN + a.OUT) * sizeof(ll);
    if (smem <= 48 * 1024) {
      dim3 grid(ceil_div(a.n_inner, MIX_NT), a.n_outer);
      mix_reg_kernel<TIn, TW, SPLIT><<<grid, MIX_NT, smem, ctx->stream>>>(a, in, Wmat, out64, hi, lo, lo2,
                                                                           ctx->skip);
      SEEMPS_LAUNCHED(ctx);
      return SEEMPS_OK;
    }
  }
  size_t smem = (((size_t)a.IN * a.OUT * sizeof(TW) + 15) & ~(size_t)15) + (size_t)a.IN * 32 * sizeof(TIn);
  if (smem > 220 * 1024) {
    seemps_set_error(ctx, "mix: MPO block %d x %d too large for shared memory", a.IN, a.OUT);
    return SEEMPS_ERR_UNSUPPORTED;
  }
  if (a.n_outer > 65535) {
    seemps_set_error(ctx, "mix: outer extent %d too large", a.n_outer);
    return SEEMPS_ERR_INVALID;
  }
  // set on every call (a cheap host call): correct for any device and thread
  if (smem > 48 * 1024)
    SEEMPS_CHECK_CUDA(ctx, cudaFuncSetAttribute(mix_kernel<TIn, TW, SPLIT>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)(220 * 1024)));
  dim3 grid(ceil_div(a.n_inner, 32), a.n_outer);
  mix_kernel<TIn, TW, SPLIT><<<grid, 256, smem, ctx->stream>>>(a, in, Wmat, out64, hi, lo, lo2, ctx->skip);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

// Wmat[i = (b, s, t)][o = (s', t', f)] = sum_e W1[b, s', s, e] W2[e, t', t, f]
__global__ void w12_kernel(const double* __restrict__ W1, const double* __restrict__ W2, int Dl,
                           int Dm, int Dr, int d, double* __restrict__ out) {
  const int d2 = d * d, IN = Dl * d2, OUT = d2 * Dr;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < IN * OUT; e += gridDim.x * blockDim.x) {
    int i = e / OUT, o = e % OUT;
    int b = i / d2, s = (i % d2) / d, t = i % d;
    int sp = o / (d * Dr), tp = (o / Dr) % d, f = o % Dr;
    double acc = 0.0;
    for (int m = 0; m < Dm; ++m)
      acc += W1[((ll)(b * d + sp) * d + s) * Dm + m] * W2[((ll)(m * d + tp) * d + t) * Dr + f];
    out[e] = acc;
  }
}

// One-site mixing matrix: Wmat[i = (b, s)][o = (s', f)] = W[b, s', s, f]
__global__ void w1_kernel(const double* __restrict__ W, int Dl, int Dr, int d, double* __restrict__ out) {
  const int IN = Dl * d, OUT = d * Dr;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < IN * OUT; e += gridDim.x * blockDim.x) {
    const int i = e / OUT, o = e % OUT;
    const int b = i / d, s = i % d, sp = o / Dr, f = o % Dr;
    out[e] = W[((ll)(b * d + sp) * d + s) * Dr + f];
  }
}

// Environment mixing matrices from W[b, s', s, f] (shape Db, d, d, Df):
//  left : Wmat[i = (s', b)][o = (f, s)]
//  right: Wmat[i = (s', f)][o = (b, s)]
__global__ void wenv_kernel(const double* __restrict__ W, int Db, int Df, int d, int right,
                            double* __restrict__ out) {
  const int IN = d * (right ? Df : Db), OUT = (right ? Db : Df) * d;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < IN * OUT; e += gridDim.x * blockDim.x) {
    int i = e / OUT, o = e % OUT;
    int sp, b, s, f;
    if (!right) {
      sp = i / Db; b = i % Db; f = o / d; s = o % d;
    } else {
      sp = i / Df; f = i % Df; b = o / d; s = o % d;
    }
    out[e] = W[((ll)(b * d + sp) * d + s) * Df + f];
  }
}

__global__ void heff_diag_kernel(const double* __restrict__ L, const double* __restrict__ W1,
                                 const double* __restrict__ W2, const double* __restrict__ R,
                                 int chil, int chir, int d, int Dl, int Dm, int Dr,
                                 double* __restrict__ diag) {
  const ll n = (ll)chil * d * d * chir;
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x) {
    int c = (int)(e % chir);
    int t = (int)((e / chir) % d);
    int s = (int)((e / ((ll)chir * d)) % d);
    int a = (int)(e / ((ll)chir * d * d));
    double acc = 0.0;
    for (int b = 0; b < Dl; ++b) {
      double lv = L[((ll)a * Dl + b) * chil + a];
      if (lv == 0.0) continue;
      for (int m = 0; m < Dm; ++m) {
        double w1 = W1[((ll)(b * d + s) * d + s) * Dm + m];
        if (w1 == 0.0) continue;
        for (int f = 0; f < Dr; ++f)
          acc += lv * w1 * W2[((ll)(m * d + t) * d + t) * Dr + f] * R[((ll)c * Dr + f) * chir + c];
      }
    }
    diag[e] = acc;
  }
}

seemps_status zero_pad_cols(seemps_ctx* ctx, __nv_bfloat16* p, int rows, int valid, int Kp) {
  if (Kp > valid && rows > 0)
    SEEMPS_CHECK_CUDA(ctx, cudaMemset2DAsync(p + valid, (size_t)Kp * 2, 0, (size_t)(Kp - valid) * 2,
                                             rows, ctx->stream));
  return SEEMPS_OK;
}

seemps_status alloc_split(seemps_ctx* ctx, ll rows, ll kp, SplitBuf* b) {
  SEEMPS_TRY(ws_alloc(ctx, (size_t)(rows * kp), &b->hi));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)(rows * kp), &b->lo));
  b->lo2 = nullptr;
  return SEEMPS_OK;
}

seemps_status alloc_split3(seemps_ctx* ctx, ll rows, ll kp, SplitBuf* b) {
  SEEMPS_TRY(alloc_split(ctx, rows, kp, b));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)(rows * kp), &b->lo2));
  return SEEMPS_OK;
}

}  // namespace

// ======================================================================== effective operator
seemps_status heff_alloc(seemps_ctx* ctx, HeffPlan* p);

seemps_status heff_plan(seemps_ctx* ctx, const seemps_pair_dims* dm, const double* L,
                        const double* W1, const double* W2, const double* R, int precision,
                        HeffPlan* p) {
  return heff_plan_braket(ctx, dm, dm->chi_l, dm->chi_r, L, W1, W2, R, precision, p);
}

seemps_status heff_plan_braket(seemps_ctx* ctx, const seemps_pair_dims* dm, int kl, int kr, const double* L,
                               const double* W1, const double* W2, const double* R, int precision,
                               HeffPlan* p) {
  const int chil = dm->chi_l, chir = dm->chi_r, d = dm->d, Dl = dm->D_l, Dm = dm->D_m, Dr = dm->D_r;
  SEEMPS_REQUIRE(ctx, chil > 0 && chir > 0 && kl > 0 && kr > 0 && d > 0 && Dl > 0 && Dm > 0 && Dr > 0,
                 "heff: non-positive dimension");
  SEEMPS_REQUIRE(ctx, L && W1 && W2 && R, "heff: null operand");
  SEEMPS_REQUIRE(ctx, precision == SEEMPS_FP64 || precision == SEEMPS_BF16X3 || precision == SEEMPS_FP64X2,
                 "heff: unknown precision %d", precision);
  p->dm = *dm;
  p->kl = kl;
  p->kr = kr;
  p->dp = d * d;
  p->precision = precision;
  p->L = L;
  p->R = R;
  const int d2 = d * d, IN = Dl * d2, OUT = d2 * Dr;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)IN * OUT, &p->Wmat));
  w12_kernel<<<stride_grid(ctx, (ll)IN * OUT, 256, 1), 256, 0, ctx->stream>>>(W1, W2, Dl, Dm, Dr, d,
                                                                                p->Wmat);
  SEEMPS_LAUNCHED(ctx);
  return heff_alloc(ctx, p);
}

// Scratch and bf16x3 operands of a plan whose dm, dp, precision, L, R and
// Wmat are set.
seemps_status heff_alloc(seemps_ctx* ctx, HeffPlan* p) {
  const int chil = p->dm.chi_l, chir = p->dm.chi_r, Dl = p->dm.D_l, Dr = p->dm.D_r;
  const int kl = p->kl, kr = p->kr;
  const int d2 = p->dp;
  const int precision = p->precision;
  const double* L = p->L;
  const double* R = p->R;
  const ll t_elems = (ll)chil * Dl * d2 * kr;  // T1[(a', b), (s, t, c)]
  const ll t2_elems = (ll)chil * d2 * Dr * kr;  // T2[(a', s', t'), (f, c)]
  if (precision == SEEMPS_FP64 || precision == SEEMPS_FP64X2) {
    const size_t parts = precision == SEEMPS_FP64X2 ? 2 : 1;  // double-FP64: hi and lo parts
    SEEMPS_TRY(ws_alloc(ctx, parts * (size_t)t_elems, &p->T1));
    SEEMPS_TRY(ws_alloc(ctx, parts * (size_t)t2_elems, &p->T2));
    return SEEMPS_OK;
  }
  p->Kp1 = (int)round_up(kl, 64);
  p->Kp3 = (int)round_up((ll)Dr * kr, 64);
  p->fuse = ctx->fuse_mix && mix_epi_ok(Dl, d2, Dr);
  SEEMPS_TRY(alloc_split(ctx, (ll)chil * Dl, p->Kp1, &p->Ls));
  SEEMPS_TRY(alloc_split(ctx, (ll)d2 * kr, p->Kp1, &p->thT));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)t_elems, &p->T1f));
  SEEMPS_TRY(alloc_split(ctx, (ll)chil * d2, p->Kp3, &p->T2s));
  SEEMPS_TRY(alloc_split(ctx, (ll)chir, p->Kp3, &p->Rs));
  // L viewed as [(a', b), a] and R as [c', (f, c)] are already K-major
  SEEMPS_TRY(split_bf16(ctx, L, kl, chil * Dl, kl, false, p->Ls.hi, p->Ls.lo));
  SEEMPS_TRY(split_bf16(ctx, R, (ll)Dr * kr, chir, Dr * kr, false, p->Rs.hi, p->Rs.lo));
  SEEMPS_TRY(zero_pad_cols(ctx, p->T2s.hi, chil * d2, Dr * kr, p->Kp3));
  SEEMPS_TRY(zero_pad_cols(ctx, p->T2s.lo, chil * d2, Dr * kr, p->Kp3));
  return SEEMPS_OK;
}

template <typename T>
seemps_status heff_run_tc(seemps_ctx* ctx, const HeffPlan* p, const T* theta, T* y);

// y = H_n theta.  Order: T1 = L . theta (sum over a), mix with W1 W2 (sum
// over b, s, t), y = T2 . R (sum over f, c).

seemps_status heff_run(seemps_ctx* ctx, const HeffPlan* p, const double* theta, double* y) {
  PhaseTimer timer(ctx, SEEMPS_PHASE_MATVEC);
  if (p->precision == SEEMPS_FP64X2) return heff_run_dd(ctx, p, theta, y);
  const int chil = p->dm.chi_l, chir = p->dm.chi_r, Dl = p->dm.D_l, Dr = p->dm.D_r;
  const int kl = p->kl, kr = p->kr;
  const int d2 = p->dp;
  MixArgs mx;
  mx.n_outer = chil;
  mx.n_inner = kr;
  mx.IN = Dl * d2;
  mx.OUT = d2 * Dr;
  mx.in_so = (ll)Dl * d2 * kr;
  mx.in_s1 = kr;
  mx.in_s2 = 0;
  mx.in_n2 = 1;
  mx.out_m2 = Dr;
  mx.out_ti = 1;
  if (p->precision == SEEMPS_FP64) {
    DgemmArgs g1 = {chil * Dl, d2 * kr, kl, 1, 1.0, 0.0,
                    p->L, kl, 1, 0, theta, (ll)d2 * kr, 1, 0, p->T1, (ll)d2 * kr, 1, 0};
    SEEMPS_TRY(dgemm(ctx, g1));
    const ll ld2 = (ll)Dr * kr;
    mx.out_so = d2 * ld2;
    mx.out_t1 = ld2;
    mx.out_t2 = kr;
    SEEMPS_TRY((launch_mix<double, double, false>(ctx, mx, p->T1, p->Wmat, p->T2, nullptr, nullptr)));
    DgemmArgs g3 = {chil * d2, chir, Dr * kr, 1, 1.0, 0.0,
                    p->T2, ld2, 1, 0, p->R, 1, ld2, 0, y, chir, 1, 0};
    return dgemm(ctx, g3);
  }
  return heff_run_tc(ctx, p, theta, y);
}

// bf16x3 on the tensor cores: theta FP64 or FP32 (split into bf16 hi/lo
// either way), y written in the same type.
template <typename T>
seemps_status heff_run_tc(seemps_ctx* ctx, const HeffPlan* p, const T* theta, T* y) {
  const int chil = p->dm.chi_l, chir = p->dm.chi_r, Dl = p->dm.D_l, Dr = p->dm.D_r;
  const int kl = p->kl, kr = p->kr;
  const int d2 = p->dp;
  SEEMPS_REQUIRE(ctx, p->precision == SEEMPS_BF16X3, "heff: the tensor-core apply needs a bf16x3 plan");
  MixArgs mx;
  mx.n_outer = chil;
  mx.n_inner = kr;
  mx.IN = Dl * d2;
  mx.OUT = d2 * Dr;
  mx.in_so = (ll)Dl * d2 * kr;
  mx.in_s1 = kr;
  mx.in_s2 = 0;
  mx.in_n2 = 1;
  mx.out_m2 = Dr;
  mx.out_ti = 1;
  SplitOperand A1 = {p->Ls.hi, p->Ls.lo, chil * Dl};
  SplitOperand B1 = {p->thT.hi, p->thT.lo, d2 * kr};
  if (p->fuse) {
    // theta's columns (s, c) become the GEMM's B rows (c, s), so that each
    // output tile holds whole (a, c) groups for the mixing in its epilogue
    SEEMPS_TRY(split_bf16_perm(ctx, theta, (ll)d2 * kr, kl, d2 * kr, kr, p->thT.hi, p->thT.lo));
    const MixEpi me = {p->Wmat, p->T2s.hi, p->T2s.lo, (ll)p->Kp3, Dl, d2, Dr, 128 / Dl, kr, chil};
    SEEMPS_TRY(tc_gemm_mix(ctx, A1, B1, p->Kp1, me));
  } else {
    SEEMPS_TRY(split_bf16(ctx, theta, (ll)d2 * kr, kl, d2 * kr, true, p->thT.hi, p->thT.lo));
    SEEMPS_TRY(tc_gemm_f32out(ctx, A1, B1, p->Kp1, p->T1f, (ll)d2 * kr));
    mx.out_so = (ll)d2 * p->Kp3;
    mx.out_t1 = p->Kp3;
    mx.out_t2 = kr;
    SEEMPS_TRY((launch_mix<float, float, true>(ctx, mx, p->T1f, p->Wmat, nullptr, p->T2s.hi, p->T2s.lo)));
  }
  SplitOperand A3 = {p->T2s.hi, p->T2s.lo, chil * d2};
  SplitOperand B3 = {p->Rs.hi, p->Rs.lo, chir};
  if constexpr (std::is_same<T, float>::value) return tc_gemm_f32out(ctx, A3, B3, p->Kp3, y, chir);
  else return tc_gemm_f64out(ctx, A3, B3, p->Kp3, y, chir);
}

seemps_status heff_run(seemps_ctx* ctx, const HeffPlan* p, const float* theta, float* y) {
  PhaseTimer timer(ctx, SEEMPS_PHASE_MATVEC);
  return heff_run_tc(ctx, p, theta, y);
}

seemps_status heff1_plan(seemps_ctx* ctx, const seemps_pair_dims* dm, const double* L, const double* W,
                         const double* R, int precision, HeffPlan* p) {
  const int chil = dm->chi_l, chir = dm->chi_r, d = dm->d, Dl = dm->D_l, Dr = dm->D_r;
  SEEMPS_REQUIRE(ctx, chil > 0 && chir > 0 && d > 0 && Dl > 0 && Dr > 0, "heff1: non-positive dimension");
  SEEMPS_REQUIRE(ctx, L && W && R, "heff1: null operand");
  SEEMPS_REQUIRE(ctx, precision == SEEMPS_FP64 || precision == SEEMPS_BF16X3,
                 "heff1: unknown precision %d", precision);
  p->dm = *dm;
  p->kl = chil;
  p->kr = chir;
  p->dp = d;
  p->precision = precision;
  p->L = L;
  p->R = R;
  const int IN = Dl * d, OUT = d * Dr;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)IN * OUT, &p->Wmat));
  w1_kernel<<<stride_grid(ctx, (ll)IN * OUT, 256, 1), 256, 0, ctx->stream>>>(W, Dl, Dr, d, p->Wmat);
  SEEMPS_LAUNCHED(ctx);
  return heff_alloc(ctx, p);
}

size_t heff_workspace_bytes(int chi, int d, int D) {
  const size_t d2 = (size_t)d * d, t = (size_t)chi * D * d2 * chi;
  const size_t kp1 = (size_t)round_up(chi, 64), kp3 = (size_t)round_up((ll)D * chi, 64);
  size_t fp64 = 4 * t * 8;  // T1, T2 with hi and lo parts (double-FP64)
  size_t mixed = 4 * ((size_t)chi * D * kp1 + d2 * chi * kp1 + (size_t)chi * d2 * kp3 + (size_t)chi * kp3) +
                 t * 4;
  size_t w = (size_t)D * d2 * d2 * D * 8;
  return (fp64 > mixed ? fp64 : mixed) + w + 16 * 256;
}

extern "C" seemps_status seemps_heff_apply(seemps_ctx* ctx, const seemps_pair_dims* dims,
                                           const double* L, const double* W1, const double* W2,
                                           const double* R, const double* theta, double* y,
                                           int precision) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, dims && theta && y, "heff_apply: null argument");
  SEEMPS_REQUIRE(ctx, theta != y, "heff_apply: y may not alias theta");
  WsFrame frame(ctx);
  HeffPlan p;
  SEEMPS_TRY(heff_plan(ctx, dims, L, W1, W2, R, precision, &p));
  return heff_run(ctx, &p, theta, y);
}

extern "C" seemps_status seemps_heff_apply_braket(seemps_ctx* ctx, const seemps_pair_dims* dims, int chib_l,
                                                  int chib_r, const double* L, const double* W1,
                                                  const double* W2, const double* R, const double* theta_b,
                                                  double* y, int precision) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, dims && theta_b && y, "heff_apply_braket: null argument");
  SEEMPS_REQUIRE(ctx, theta_b != y, "heff_apply_braket: y may not alias theta_b");
  WsFrame frame(ctx);
  HeffPlan p;
  SEEMPS_TRY(heff_plan_braket(ctx, dims, chib_l, chib_r, L, W1, W2, R, precision, &p));
  return heff_run(ctx, &p, theta_b, y);
}

extern "C" seemps_status seemps_heff1_apply(seemps_ctx* ctx, const seemps_pair_dims* dims, const double* L,
                                            const double* W, const double* R, const double* A, double* y,
                                            int precision) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, dims && A && y, "heff1_apply: null argument");
  SEEMPS_REQUIRE(ctx, A != y, "heff1_apply: y may not alias A");
  WsFrame frame(ctx);
  HeffPlan p;
  SEEMPS_TRY(heff1_plan(ctx, dims, L, W, R, precision, &p));
  return heff_run(ctx, &p, A, y);
}

extern "C" seemps_status seemps_heff_diagonal(seemps_ctx* ctx, const seemps_pair_dims* dm,
                                              const double* L, const double* W1, const double* W2,
                                              const double* R, double* diag) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, dm && L && W1 && W2 && R && diag, "heff_diagonal: null argument");
  const ll n = (ll)dm->chi_l * dm->d * dm->d * dm->chi_r;
  SEEMPS_REQUIRE(ctx, n > 0, "heff_diagonal: empty problem");
  heff_diag_kernel<<<stride_grid(ctx, n, 256, 8), 256, 0, ctx->stream>>>(
      L, W1, W2, R, dm->chi_l, dm->chi_r, dm->d, dm->D_l, dm->D_m, dm->D_r, diag);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

// ======================================================================== environments
size_t env_workspace_bytes(int chi, int d, int D) {
  const size_t x = (size_t)chi * D * d * chi;
  const size_t kpa = (size_t)round_up(chi, 64), kpb = (size_t)round_up((ll)chi * d, 64);
  size_t fp64 = 4 * x * 8;  // X1, Z with hi and lo parts (double-FP64)
  size_t mixed = 6 * ((size_t)d * chi * kpa + (size_t)D * chi * kpa + (size_t)chi * D * kpb +
                      (size_t)chi * kpb) + x * 4;  // three bf16 planes per operand
  return (fp64 > mixed ? fp64 : mixed) + (size_t)D * D * d * d * 8 + 16 * 256;
}

extern "C" seemps_status seemps_env_update(seemps_ctx* ctx, int side, int chi_in, int chi_out,
                                           int d, int D_in, int D_out, const double* E_in,
                                           const double* A, const double* W, double* E_out,
                                           int precision) {
  return env_update_braket(ctx, side, chi_in, chi_in, chi_out, chi_out, d, D_in, D_out, E_in, A, A, W, E_out,
                           precision);
}

extern "C" seemps_status seemps_env_update_braket(seemps_ctx* ctx, int side, int chi_in_x, int chi_in_b,
                                                  int chi_out_x, int chi_out_b, int d, int D_in, int D_out,
                                                  const double* E_in, const double* X, const double* B,
                                                  const double* W, double* E_out, int precision) {
  return env_update_braket(ctx, side, chi_in_x, chi_in_b, chi_out_x, chi_out_b, d, D_in, D_out, E_in, X, B, W,
                           E_out, precision);
}

// E_out from E_in, the bra tensor X, the MPO tensor W and the ket tensor B:
// X1 = (bra contraction of E_in), mix with W, E_out = (ket contraction).
seemps_status env_update_braket(seemps_ctx* ctx, int side, int cix, int cib, int cox, int cob, int d, int D_in,
                                int D_out, const double* E_in, const double* X, const double* B,
                                const double* W, double* E_out, int precision) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, E_in && X && B && W && E_out, "env_update: null argument");
  SEEMPS_REQUIRE(ctx, cix > 0 && cib > 0 && cox > 0 && cob > 0 && d > 0 && D_in > 0 && D_out > 0,
                 "env_update: non-positive dimension");
  SEEMPS_REQUIRE(ctx, side == SEEMPS_LEFT || side == SEEMPS_RIGHT, "env_update: bad side");
  SEEMPS_REQUIRE(ctx, precision == SEEMPS_FP64 || precision == SEEMPS_BF16X3 || precision == SEEMPS_FP64X2,
                 "env_update: unknown precision");
  WsFrame frame(ctx);
  PhaseTimer timer(ctx, SEEMPS_PHASE_ENV);
  const int Di = D_in, Do = D_out;
  const bool right = (side == SEEMPS_RIGHT);
  // mixing matrix
  double* Wmat;
  const int IN = d * Di, OUT = Do * d;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)IN * OUT, &Wmat));
  if (!right)
    wenv_kernel<<<stride_grid(ctx, (ll)IN * OUT, 256, 1), 256, 0, ctx->stream>>>(W, Di, Do, d, 0, Wmat);
  else
    wenv_kernel<<<stride_grid(ctx, (ll)IN * OUT, 256, 1), 256, 0, ctx->stream>>>(W, Do, Di, d, 1, Wmat);
  SEEMPS_LAUNCHED(ctx);

  MixArgs mx;
  mx.IN = IN;
  mx.OUT = OUT;
  const ll xrows = (ll)d * cox, xcols = (ll)Di * cib;  // X1 is [xrows x xcols] in both cases
  const ll zcols = (ll)cib * d;                        // Z is [cox*Do x zcols]
  if (!right) {
    // X1[(s', c'), (b, a)] -> Z[(c', f), (a, s)]; outer c', inner a
    mx.n_outer = cox;
    mx.n_inner = cib;
    mx.in_so = xcols;
    mx.in_n2 = Di;
    mx.in_s1 = (ll)cox * xcols;
    mx.in_s2 = cib;
    mx.out_m2 = d;
    mx.out_t2 = 1;
    mx.out_ti = d;
  } else {
    // X1[(a', s'), (f, c)] -> Z[(a', b), (s, c)]; outer a', inner c
    mx.n_outer = cox;
    mx.n_inner = cib;
    mx.in_so = (ll)d * xcols;
    mx.in_n2 = Di;
    mx.in_s1 = xcols;
    mx.in_s2 = cib;
    mx.out_m2 = d;
    mx.out_t2 = cib;
    mx.out_ti = 1;
  }
  if (precision == SEEMPS_FP64X2)
    return env_update_dd(ctx, side, cix, cib, cox, cob, d, Di, Do, E_in, X, B, Wmat, mx, E_out);
  if (precision == SEEMPS_FP64) {
    double *X1, *Z;
    SEEMPS_TRY(ws_alloc(ctx, (size_t)(xrows * xcols), &X1));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)((ll)cox * Do * zcols), &Z));
    if (!right) {
      DgemmArgs g1 = {d * cox, Di * cib, cix, 1, 1.0, 0.0, X, 1, (ll)d * cox, 0,
                      E_in, xcols, 1, 0, X1, xcols, 1, 0};
      SEEMPS_TRY(dgemm(ctx, g1));
    } else {
      DgemmArgs g1 = {cox * d, Di * cib, cix, 1, 1.0, 0.0, X, cix, 1, 0,
                      E_in, xcols, 1, 0, X1, xcols, 1, 0};
      SEEMPS_TRY(dgemm(ctx, g1));
    }
    mx.out_so = (ll)Do * zcols;
    mx.out_t1 = zcols;
    SEEMPS_TRY((launch_mix<double, double, false>(ctx, mx, X1, Wmat, Z, nullptr, nullptr)));
    if (!right) {
      DgemmArgs g2 = {cox * Do, cob, cib * d, 1, 1.0, 0.0, Z, zcols, 1, 0,
                      B, cob, 1, 0, E_out, cob, 1, 0};
      return dgemm(ctx, g2);
    }
    DgemmArgs g2 = {cox * Do, cob, d * cib, 1, 1.0, 0.0, Z, zcols, 1, 0,
                    B, 1, (ll)d * cib, 0, E_out, cob, 1, 0};
    return dgemm(ctx, g2);
  }
  // bf16x3 sweep: the environment is renewed ~N times per sweep from the
  // previous one, so its products carry three bf16 planes (six products,
  // ~2^-24 relative error) instead of two: their errors would otherwise
  // accumulate over the chain to ~1e-4 of the energy.  The update is a small
  // share of a pair update.
  const int kpa = (int)round_up(cix, 64), kpz = (int)round_up(zcols, 64);
  SplitBuf a1, e1, z, a2;
  float* X1;
  SEEMPS_TRY(alloc_split3(ctx, xrows, kpa, &a1));
  SEEMPS_TRY(alloc_split3(ctx, xcols, kpa, &e1));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)(xrows * xcols), &X1));
  SEEMPS_TRY(alloc_split3(ctx, (ll)cox * Do, kpz, &z));
  SEEMPS_TRY(alloc_split3(ctx, cob, kpz, &a2));
  if (!right) {
    // Xt = (X viewed [cix x d cox])^T, Lt = (E viewed [cix x Di cib])^T, Bt = (B viewed [cib d x cob])^T
    SEEMPS_TRY(split_bf16_3(ctx, X, (ll)d * cox, cix, d * cox, true, a1.hi, a1.lo, a1.lo2));
    SEEMPS_TRY(split_bf16_3(ctx, E_in, xcols, cix, Di * cib, true, e1.hi, e1.lo, e1.lo2));
    SEEMPS_TRY(split_bf16_3(ctx, B, cob, cib * d, cob, true, a2.hi, a2.lo, a2.lo2));
  } else {
    // X viewed [cox d x cix] (K-major), Rt = (E viewed [cix x Di cib])^T, B viewed [cob x d cib]
    SEEMPS_TRY(split_bf16_3(ctx, X, cix, cox * d, cix, false, a1.hi, a1.lo, a1.lo2));
    SEEMPS_TRY(split_bf16_3(ctx, E_in, xcols, cix, Di * cib, true, e1.hi, e1.lo, e1.lo2));
    SEEMPS_TRY(split_bf16_3(ctx, B, (ll)d * cib, cob, d * cib, false, a2.hi, a2.lo, a2.lo2));
  }
  SplitOperand opA1 = {a1.hi, a1.lo, (int)xrows, a1.lo2};
  SplitOperand opB1 = {e1.hi, e1.lo, (int)xcols, e1.lo2};
  SEEMPS_TRY(tc_gemm_f32out(ctx, opA1, opB1, kpa, X1, xcols));
  SEEMPS_TRY(zero_pad_cols(ctx, z.hi, cox * Do, (int)zcols, kpz));
  SEEMPS_TRY(zero_pad_cols(ctx, z.lo, cox * Do, (int)zcols, kpz));
  SEEMPS_TRY(zero_pad_cols(ctx, z.lo2, cox * Do, (int)zcols, kpz));
  mx.out_so = (ll)Do * kpz;
  mx.out_t1 = kpz;
  SEEMPS_TRY((launch_mix<float, float, true>(ctx, mx, X1, Wmat, nullptr, z.hi, z.lo, z.lo2)));
  SplitOperand opA2 = {z.hi, z.lo, cox * Do, z.lo2};
  SplitOperand opB2 = {a2.hi, a2.lo, cob, a2.lo2};
  return tc_gemm_f64out(ctx, opA2, opB2, kpz, E_out, cob);
}

extern "C" seemps_status seemps_env_update_linear(seemps_ctx* ctx, int side, int chi_in,
                                                  int chi_out, int chib_in, int chib_out, int d,
                                                  const double* F_in, const double* A,
                                                  const double* B, double* F_out) {
  return env_update_linear_run(ctx, side, chi_in, chi_out, chib_in, chib_out, d, F_in, A, B, F_out, SEEMPS_FP64);
}

seemps_status env_update_linear_run(seemps_ctx* ctx, int side, int chi_in, int chi_out, int chib_in, int chib_out,
                                    int d, const double* F_in, const double* A, const double* B, double* F_out,
                                    int precision) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, F_in && A && B && F_out, "env_update_linear: null argument");
  SEEMPS_REQUIRE(ctx, chi_in > 0 && chi_out > 0 && chib_in > 0 && chib_out > 0 && d > 0,
                 "env_update_linear: non-positive dimension");
  WsFrame frame(ctx);
  const int ci = chi_in, co = chi_out, bi = chib_in, bo = chib_out;
  double* T;
  if (side == SEEMPS_LEFT) {
    // T[a, (s, c'')] = F[a, a''] B[a'', (s, c'')]; F_out[c, c''] = sum_(a,s) A[(a,s), c] T[(a,s), c'']
    SEEMPS_TRY(ws_alloc(ctx, (size_t)ci * d * bo, &T));
    DgemmArgs g1 = {ci, d * bo, bi, 1, 1.0, 0.0, F_in, bi, 1, 0, B, (ll)d * bo, 1, 0, T, (ll)d * bo, 1, 0};
    SEEMPS_TRY(gemm_prec(ctx, g1, precision));
    DgemmArgs g2 = {co, bo, ci * d, 1, 1.0, 0.0, A, 1, co, 0, T, bo, 1, 0, F_out, bo, 1, 0};
    return gemm_prec(ctx, g2, precision);
  }
  SEEMPS_REQUIRE(ctx, side == SEEMPS_RIGHT, "env_update_linear: bad side");
  // T[(a'', s), c] = sum_c'' B[(a'', s), c''] G[c, c'']; G_out[a, a''] = sum_(s,c) A[a, (s,c)] T[a'', (s,c)]
  SEEMPS_TRY(ws_alloc(ctx, (size_t)bo * d * ci, &T));
  DgemmArgs g1 = {bo * d, ci, bi, 1, 1.0, 0.0, B, bi, 1, 0, F_in, 1, bi, 0, T, ci, 1, 0};
  SEEMPS_TRY(gemm_prec(ctx, g1, precision));
  DgemmArgs g2 = {co, bo, d * ci, 1, 1.0, 0.0, A, (ll)d * ci, 1, 0, T, 1, (ll)d * ci, 0, F_out, bo, 1, 0};
  return gemm_prec(ctx, g2, precision);
}

extern "C" seemps_status seemps_b_effective(seemps_ctx* ctx, int chi_l, int chi_r, int chib_l,
                                            int chib_m, int chib_r, int d, const double* F,
                                            const double* B1, const double* B2, const double* G,
                                            double* b) {
  return b_effective_run(ctx, chi_l, chi_r, chib_l, chib_m, chib_r, d, F, B1, B2, G, b, SEEMPS_FP64);
}

seemps_status b_effective_run(seemps_ctx* ctx, int chi_l, int chi_r, int chib_l, int chib_m, int chib_r, int d,
                              const double* F, const double* B1, const double* B2, const double* G, double* b,
                              int precision) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, F && B1 && B2 && G && b, "b_effective: null argument");
  SEEMPS_REQUIRE(ctx, chi_l > 0 && chi_r > 0 && chib_l > 0 && chib_m > 0 && chib_r > 0 && d > 0,
                 "b_effective: non-positive dimension");
  WsFrame frame(ctx);
  double *T1, *T2;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)chi_l * d * chib_m, &T1));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)chi_l * d * d * chib_r, &T2));
  DgemmArgs g1 = {chi_l, d * chib_m, chib_l, 1, 1.0, 0.0, F, chib_l, 1, 0, B1, (ll)d * chib_m, 1, 0,
                  T1, (ll)d * chib_m, 1, 0};
  SEEMPS_TRY(gemm_prec(ctx, g1, precision));
  DgemmArgs g2 = {chi_l * d, d * chib_r, chib_m, 1, 1.0, 0.0, T1, chib_m, 1, 0, B2, (ll)d * chib_r, 1, 0,
                  T2, (ll)d * chib_r, 1, 0};
  SEEMPS_TRY(gemm_prec(ctx, g2, precision));
  DgemmArgs g3 = {chi_l * d * d, chi_r, chib_r, 1, 1.0, 0.0, T2, chib_r, 1, 0, G, 1, chib_r, 0,
                  b, chi_r, 1, 0};
  return gemm_prec(ctx, g3, precision);
}

// One GEMM C = A B (alpha 1, beta 0, no batch) in the given precision: the
// FP64 CUDA-core GEMM, or for BF16X3 the tensor-core GEMM with each operand
// split into K-major bf16 hi/lo planes (either storage order of A, B and C:
// a column-major C is formed as C^T = B^T A^T).  Other argument patterns
// fall back to the FP64 GEMM.
seemps_status gemm_prec(seemps_ctx* ctx, const DgemmArgs& g, int precision) {
  const bool plain = g.batch == 1 && g.alpha == 1.0 && g.beta == 0.0;
  const bool a_rm = g.sAk == 1, a_cm = g.sAm == 1;
  const bool b_rm = g.sBn == 1, b_cm = g.sBk == 1;
  const bool c_rm = g.sCn == 1, c_cm = g.sCm == 1;
  if (precision != SEEMPS_BF16X3 || !plain || !(a_rm || a_cm) || !(b_rm || b_cm) || !(c_rm || c_cm) ||
      !tc_available(ctx))
    return dgemm(ctx, g);
  WsFrame frame(ctx);
  const int Kp = (int)round_up(g.K, 64);
  SplitBuf a, b;
  SEEMPS_TRY(alloc_split(ctx, g.M, Kp, &a));
  SEEMPS_TRY(alloc_split(ctx, g.N, Kp, &b));
  // A as [M x Kp] K-major
  if (a_rm) SEEMPS_TRY(split_bf16(ctx, g.A, g.sAm, g.M, g.K, false, a.hi, a.lo));
  else SEEMPS_TRY(split_bf16(ctx, g.A, g.sAk, g.K, g.M, true, a.hi, a.lo));
  // B as [N x Kp] K-major
  if (b_rm) SEEMPS_TRY(split_bf16(ctx, g.B, g.sBk, g.K, g.N, true, b.hi, b.lo));
  else SEEMPS_TRY(split_bf16(ctx, g.B, g.sBn, g.N, g.K, false, b.hi, b.lo));
  SplitOperand oa = {a.hi, a.lo, g.M};
  SplitOperand ob = {b.hi, b.lo, g.N};
  if (c_rm) return tc_gemm_f64out(ctx, oa, ob, Kp, g.C, g.sCm);
  return tc_gemm_f64out(ctx, ob, oa, Kp, g.C, g.sCn);
}

// The two-site vector in the sweep's precision: FP64 GEMM, or for BF16X3 the
// tensor-core GEMM  theta[(a,s),(t,c)] = sum_m A1[(a,s), m] A2[m, (t,c)]  with A1
// K-major as stored and A2 split transposed.
seemps_status two_site_run(seemps_ctx* ctx, int chi_l, int chi_m, int chi_r, int d, const double* A1,
                           const double* A2, double* theta, int precision) {
  if (precision != SEEMPS_BF16X3 || !tc_available(ctx))
    return seemps_two_site(ctx, chi_l, chi_m, chi_r, d, A1, A2, theta);
  WsFrame frame(ctx);
  const int M = chi_l * d, N = d * chi_r, K = chi_m;
  const int Kp = (int)round_up(K, 64);
  SplitBuf a, b;
  SEEMPS_TRY(alloc_split(ctx, M, Kp, &a));
  SEEMPS_TRY(alloc_split(ctx, N, Kp, &b));
  SEEMPS_TRY(split_bf16(ctx, A1, K, M, K, false, a.hi, a.lo));
  SEEMPS_TRY(split_bf16(ctx, A2, N, K, N, true, b.hi, b.lo));
  SplitOperand oa = {a.hi, a.lo, M};
  SplitOperand ob = {b.hi, b.lo, N};
  return tc_gemm_f64out(ctx, oa, ob, Kp, theta, N);
}

extern "C" seemps_status seemps_two_site(seemps_ctx* ctx, int chi_l, int chi_m, int chi_r, int d,
                                         const double* A1, const double* A2, double* theta) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, A1 && A2 && theta, "two_site: null argument");
  SEEMPS_REQUIRE(ctx, chi_l > 0 && chi_m > 0 && chi_r > 0 && d > 0, "two_site: non-positive dimension");
  DgemmArgs g = {chi_l * d, d * chi_r, chi_m, 1, 1.0, 0.0, A1, chi_m, 1, 0, A2, (ll)d * chi_r, 1, 0,
                 theta, (ll)d * chi_r, 1, 0};
  return dgemm(ctx, g);
}
