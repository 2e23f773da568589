// Shared infrastructure of the sweep library: the context, the workspace
// stack, error reporting and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "../../include/seemps_gb300.h"

typedef long long ll;

// Bounded device waits give up after this many SM clocks (about 1 s at 2 GHz)
// and record SEEMPS_ERR_TIMEOUT in the status word.
#define SEEMPS_WAIT_CLOCKS (2000000000LL)

// Upper bound on the Jacobi sweeps of one SVD call.
#define SEEMPS_MAX_JACOBI_SWEEPS 256

struct seemps_ctx {
  int device;
  cudaStream_t stream;
  char* ws;              // caller-owned device workspace
  size_t ws_bytes;
  size_t ws_top;         // stack pointer of the workspace
  int* d_status;         // device status word (first bytes of the workspace)
  double* d_scalars;     // 32 device doubles of scratch scalars
  int* h_status;         // pinned host copy for seemps_device_status
  // Optional device flag: while set (non-null and *skip != 0) the kernels of
  // the matvec chain return at once.  The local solvers point it at their
  // "converged / broke down" word so that work queued past the stopping
  // point costs only launch overhead.
  const int* skip;
  // per-phase CUDA-event timing (timing.cuh)
  int timing;
  int ev_used;
  cudaEvent_t ev[512];
  int ev_phase[256];
  double phase_ms[SEEMPS_PHASE_COUNT];
  long long phase_n[SEEMPS_PHASE_COUNT];
  int sm_count;
  int cc_major, cc_minor;
  long long launches;
  // limit (SM clocks) of the software waits: grid barriers and block
  // hand-offs of the cooperative Jacobi kernels (SEEMPS_WAIT_CLOCKS unless
  // seemps_set_wait_limit changed it)
  long long wait_clocks;
  // the effective operator's MPO mixing in the first GEMM's epilogue
  int fuse_mix;
  // tile autotuner (tc_gemm.cu): use recorded winners; counters of lookups
  int autotune;
  long long tune_hits, tune_shapes;
  // Jacobi SVD counters (large-problem path): calls, sweeps, pair visits and
  // algorithmic FP32 operations (see seemps_svd_stats)
  long long svd_calls, svd_sweeps, svd_pairs;
  double svd_flops;
  // per-sweep rotations / visits of the most recent such call
  int svd_last_n;
  int svd_last_rot[SEEMPS_MAX_JACOBI_SWEEPS], svd_last_vis[SEEMPS_MAX_JACOBI_SWEEPS];
  // cleanup phase of that kernel (see seemps_svd_cleanup_stats)
  long long svd_cleanup_calls, svd_cleanup_rounds, svd_cleanup_fallbacks;
  char err[512];
};

// ----------------------------------------------------------------- errors
void seemps_set_error(seemps_ctx* ctx, const char* fmt, ...);

#define SEEMPS_CHECK_CUDA(ctx, expr)                                              \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      seemps_set_error(ctx, "%s:%d: %s: %s", __FILE__, __LINE__, #expr,           \
                       cudaGetErrorString(_e));                                   \
      return SEEMPS_ERR_CUDA;                                                     \
    }                                                                             \
  } while (0)

// Call after every kernel launch: counts the launch and checks launch errors.
#define SEEMPS_LAUNCHED(ctx)                                                      \
  do {                                                                            \
    (ctx)->launches++;                                                            \
    cudaError_t _e = cudaGetLastError();                                          \
    if (_e != cudaSuccess) {                                                      \
      seemps_set_error(ctx, "%s:%d: kernel launch: %s", __FILE__, __LINE__,       \
                       cudaGetErrorString(_e));                                   \
      return SEEMPS_ERR_CUDA;                                                     \
    }                                                                             \
  } while (0)

#define SEEMPS_TRY(expr)                                                          \
  do {                                                                            \
    seemps_status _s = (expr);                                                    \
    if (_s != SEEMPS_OK) return _s;                                               \
  } while (0)

#define SEEMPS_REQUIRE(ctx, cond, ...)                                            \
  do {                                                                            \
    if (!(cond)) {                                                                \
      seemps_set_error(ctx, __VA_ARGS__);                                         \
      return SEEMPS_ERR_INVALID;                                                  \
    }                                                                             \
  } while (0)

// ----------------------------------------------------------------- workspace
// A stack: every entry point records the top on entry (WsFrame) and pops
// back on exit, so nested calls (sweep -> local solver -> matvec) share the
// buffer without fragmentation.
struct WsFrame {
  seemps_ctx* ctx;
  size_t saved;
  explicit WsFrame(seemps_ctx* c) : ctx(c), saved(c->ws_top) {}
  ~WsFrame() { ctx->ws_top = saved; }
};

template <typename T>
static inline seemps_status ws_alloc(seemps_ctx* ctx, size_t count, T** out) {
  size_t bytes = count * sizeof(T);
  size_t start = (ctx->ws_top + 255) & ~(size_t)255;
  if (start + bytes > ctx->ws_bytes) {
    seemps_set_error(ctx, "workspace too small: need %zu more bytes (have %zu, used %zu)",
                     bytes, ctx->ws_bytes, start);
    return SEEMPS_ERR_WORKSPACE;
  }
  *out = reinterpret_cast<T*>(ctx->ws + start);
  ctx->ws_top = start + bytes;
  return SEEMPS_OK;
}

static inline int ceil_div(ll a, ll b) { return (int)((a + b - 1) / b); }
static inline ll round_up(ll a, ll b) { return ((a + b - 1) / b) * b; }

// Grid sizes for grid-stride kernels: a multiple of the SM count.
static inline int stride_grid(const seemps_ctx* ctx, ll n, int threads, int per_sm = 4) {
  ll want = (n + threads - 1) / threads;
  ll cap = (ll)ctx->sm_count * per_sm;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

// ----------------------------------------------------------------- device helpers
__device__ __forceinline__ void post_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum for blockDim.x a multiple of 32 (<= 1024); every thread
// receives the total.  `sh` needs 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// Lane index whose warp total rs_reduce returns: the low log2(NV) lane bits
// reversed.
template <int NV>
static __device__ __forceinline__ int rs_index(int lane) {
  int idx = 0;
#pragma unroll
  for (int m = 1, h = NV / 2; h >= 1; m <<= 1, h >>= 1)
    if (lane & m) idx += h;
  return idx;
}

// Warp reduce-scatter of NV values (NV a power of two <= 32): every lane gets
// the warp total of value rs_index<NV>(lane).  At each halving level a lane
// keeps one half of its values and adds the partner's copy of that half.
template <int NV>
static __device__ __forceinline__ float rs_reduce(float (&x)[NV], int lane) {
  float cur[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) cur[j] = x[j];
#pragma unroll
  for (int m = 1, n = NV; n > 1; m <<= 1, n >>= 1) {
    const bool up = (lane & m) != 0;
#pragma unroll
    for (int j = 0; j < n / 2; ++j) {
      const float keep = up ? cur[j + n / 2] : cur[j];
      const float send = up ? cur[j] : cur[j + n / 2];
      cur[j] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  float t = cur[0];
#pragma unroll
  for (int m = NV; m < 32; m <<= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
  return t;
}

// ----------------------------------------------------------------- internal API
// FP64 CUDA-core GEMM with arbitrary element strides:
//   C[b](m, n) = alpha * sum_k A[b](m, k) B[b](k, n) + beta * C[b](m, n)
// with X(i, j) at X + b * bsX + i * sX0 + j * sX1.
struct DgemmArgs {
  int M, N, K, batch;
  double alpha, beta;
  const double* A; ll sAm, sAk, bsA;
  const double* B; ll sBk, sBn, bsB;
  double* C; ll sCm, sCn, bsC;
  const int* skip;  // filled in by dgemm() from the context
};
seemps_status dgemm(seemps_ctx* ctx, const DgemmArgs& a);

// Split-precision (bf16x3) tensor-core GEMM, both operands K-major:
//   C(m, n) = sum_k A(m, k) B(n, k),  A = A_hi + A_lo, B = B_hi + B_lo,
// computed as A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation.
// A_* are [M x Kp], B_* are [N x Kp] bf16 row-major with Kp a multiple of 64
// (the caller zero-fills the padding).  C is fp32 or fp64 with row stride ldc.
// With a third plane lo2 on both operands (a = hi + lo + lo2, each bf16,
// the split of a to about 2^-24) the GEMM forms six products: hi hi, hi lo,
// lo hi, hi lo2, lo lo, lo2 hi (relative error near 2^-24; 128-wide tiles).
struct SplitOperand {
  const __nv_bfloat16* hi;
  const __nv_bfloat16* lo;
  int rows;
  const __nv_bfloat16* lo2 = nullptr;
};
seemps_status tc_gemm_f32out(seemps_ctx* ctx, const SplitOperand& A, const SplitOperand& B, int Kp,
                             float* C, ll ldc);
seemps_status tc_gemm_f64out(seemps_ctx* ctx, const SplitOperand& A, const SplitOperand& B, int Kp,
                             double* C, ll ldc);
bool tc_available(seemps_ctx* ctx);

// The effective operator's MPO mixing, done by the first GEMM's epilogue:
// for each (a, c) the tile's T1[(a, w), (c, s)] (w < Dl, s < d2) form the
// inputs i = w d2 + s of out[o] = sum_i W[i][o] T1_i, o = s' Dr + w_r, which
// is split into bf16 hi/lo at row a d2 + s', column w_r kr + c of the
// second GEMM's A operand (row stride ldo).  The GEMM's A rows are (a, w)
// and its B rows (c, s); every M tile holds apt whole groups of Dl rows.
struct MixEpi {
  const double* W;  // Dl d2 x d2 Dr
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
  ll ldo;
  int Dl, d2, Dr, apt, kr, chil;
};
// Whether the fused path applies: d2 a power of two <= 16, Dl d2 and d2 Dr <= 32,
// and 128-row tiles lose at most 1/8 of their rows to whole Dl groups.
bool mix_epi_ok(int Dl, int d2, int Dr);
// T1 = A B^T (A: chil Dl rows, B: d2 kr rows ordered (c, s)) and the mixing
// above, in one persistent launch.
seemps_status tc_gemm_mix(seemps_ctx* ctx, const SplitOperand& A, const SplitOperand& B, int Kp,
                          const MixEpi& mx);

// Split an fp64 or fp32 [R x C] matrix (row stride ld) into bf16 hi/lo.
//   transpose = false: out [R x Cp] (Cp = round_up(C, 64), zero padded)
//   transpose = true : out [C x Rp] (Rp = round_up(R, 64), zero padded)
seemps_status split_bf16(seemps_ctx* ctx, const double* in, ll ld, int R, int C, bool transpose,
                         __nv_bfloat16* hi, __nv_bfloat16* lo);
seemps_status split_bf16(seemps_ctx* ctx, const float* in, ll ld, int R, int C, bool transpose,
                         __nv_bfloat16* hi, __nv_bfloat16* lo);
// Transposing split whose output rows are permuted: input column
// s kr + c (s < C / kr) becomes output row c (C / kr) + s.
seemps_status split_bf16_perm(seemps_ctx* ctx, const double* in, ll ld, int R, int C, int kr,
                              __nv_bfloat16* hi, __nv_bfloat16* lo);
seemps_status split_bf16_perm(seemps_ctx* ctx, const float* in, ll ld, int R, int C, int kr,
                              __nv_bfloat16* hi, __nv_bfloat16* lo);
// The same into three planes hi, lo, lo2 (a = hi + lo + lo2 to ~2^-24 |a|).
seemps_status split_bf16_3(seemps_ctx* ctx, const double* in, ll ld, int R, int C, bool transpose,
                           __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2);

// FP32 Householder QR of the column-major M x N matrix A (destroyed), R
// factor only; X receives R^T as k = min(M, N) columns of length N
// (X[j][c] = R(j, c), zero for c < j).  qr_supported tells whether M fits
// the panel kernel (M <= 4096).
bool qr_supported(int M, int N);
seemps_status qr_r_transpose(seemps_ctx* ctx, float* A, int M, int N, float* X);

// Workspace bytes of the individual pieces (used by seemps_workspace_bytes).
size_t heff_workspace_bytes(int chi, int d, int D);
size_t env_workspace_bytes(int chi, int d, int D);
size_t svd_workspace_bytes(int m, int n);
size_t lanczos_workspace_bytes(int chi, int d, int D, int k);
size_t pcg_workspace_bytes(int chi, int d, int D);

// Device-pointer energy/rank helpers shared by the sweep.
seemps_status copy_scalar_to_host(seemps_ctx* ctx, const void* dptr, void* hptr, size_t bytes);
