// Context, workspace sizing, status reporting, and the FP64 CUDA-core GEMM
// used by the FP64 path of every contraction.
#include <stdarg.h>
#include <stdlib.h>

#include "common.cuh"
#include "timing.cuh"

void seemps_set_error(seemps_ctx* ctx, const char* fmt, ...) {
  if (!ctx || ctx->err[0]) return;  // keep the first error
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
  va_end(ap);
}

extern "C" seemps_status seemps_create(seemps_ctx** out, int device, void* stream, void* workspace,
                                       size_t workspace_bytes) {
  if (!out) return SEEMPS_ERR_INVALID;
  *out = nullptr;
  if (!workspace || workspace_bytes < 4096 || ((uintptr_t)workspace & 255)) return SEEMPS_ERR_INVALID;
  seemps_ctx* ctx = (seemps_ctx*)calloc(1, sizeof(seemps_ctx));
  if (!ctx) return SEEMPS_ERR_INVALID;
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  ctx->ws = (char*)workspace;
  ctx->ws_bytes = workspace_bytes;
  if (cudaSetDevice(device) != cudaSuccess) {
    free(ctx);
    return SEEMPS_ERR_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    free(ctx);
    return SEEMPS_ERR_CUDA;
  }
  ctx->sm_count = prop.multiProcessorCount;
  ctx->wait_clocks = SEEMPS_WAIT_CLOCKS;
  ctx->fuse_mix = 0;
  ctx->cc_major = prop.major;
  ctx->cc_minor = prop.minor;
  // first 256 bytes: status word; next 256: 32 scratch doubles
  ctx->d_status = (int*)ctx->ws;
  ctx->d_scalars = (double*)(ctx->ws + 256);
  ctx->ws_top = 512;
  if (cudaMallocHost((void**)&ctx->h_status, sizeof(int)) != cudaSuccess) {
    free(ctx);
    return SEEMPS_ERR_CUDA;
  }
  if (cudaMemsetAsync(ctx->ws, 0, 512, ctx->stream) != cudaSuccess) {
    cudaFreeHost(ctx->h_status);
    free(ctx);
    return SEEMPS_ERR_CUDA;
  }
  *out = ctx;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_destroy(seemps_ctx* ctx) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  cudaStreamSynchronize(ctx->stream);
  for (int i = 0; i < 512; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  free(ctx);
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_set_stream(seemps_ctx* ctx, void* stream) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  ctx->stream = (cudaStream_t)stream;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_set_fused_mixing(seemps_ctx* ctx, int enabled) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  ctx->fuse_mix = enabled ? 1 : 0;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_set_wait_limit(seemps_ctx* ctx, long long clocks) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  if (clocks < 0 || clocks > SEEMPS_WAIT_CLOCKS) clocks = SEEMPS_WAIT_CLOCKS;
  ctx->wait_clocks = clocks;
  return SEEMPS_OK;
}

extern "C" const char* seemps_last_error(const seemps_ctx* ctx) {
  return ctx ? ctx->err : "null context";
}

extern "C" seemps_status seemps_launch_count(const seemps_ctx* ctx, long long* count_out) {
  if (!ctx || !count_out) return SEEMPS_ERR_INVALID;
  *count_out = ctx->launches;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_device_status(seemps_ctx* ctx, int* status_out) {
  if (!ctx || !status_out) return SEEMPS_ERR_INVALID;
  SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int),
                                         cudaMemcpyDeviceToHost, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *status_out = *ctx->h_status;
  return SEEMPS_OK;
}

// ----------------------------------------------------------------- timing
static bool timing_any_open(const seemps_ctx* ctx) {
  for (int i = 0; i < ctx->ev_used; ++i)
    if (!(ctx->ev_phase[i] & 0x100)) return true;
  return false;
}

int timing_begin(seemps_ctx* ctx, int phase) {
  if (!ctx->timing) return -1;
  if (ctx->ev_used >= 256) {
    // the pool is full: drain it if no enclosing phase is still open,
    // otherwise leave this interval untimed
    if (timing_any_open(ctx) || timing_flush(ctx) != SEEMPS_OK) return -1;
  }
  const int slot = ctx->ev_used++;
  for (int k = 0; k < 2; ++k)
    if (!ctx->ev[2 * slot + k] && cudaEventCreate(&ctx->ev[2 * slot + k]) != cudaSuccess) return -1;
  ctx->ev_phase[slot] = phase;
  cudaEventRecord(ctx->ev[2 * slot], ctx->stream);
  return slot;
}

void timing_end(seemps_ctx* ctx, int slot) {
  if (slot < 0) return;
  cudaEventRecord(ctx->ev[2 * slot + 1], ctx->stream);
  ctx->ev_phase[slot] |= 0x100;  // closed
}

// Accumulates every recorded interval; does nothing while a phase is open.
seemps_status timing_flush(seemps_ctx* ctx) {
  if (ctx->ev_used == 0 || timing_any_open(ctx)) return SEEMPS_OK;
  SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < ctx->ev_used; ++i) {
    float ms = 0.f;
    SEEMPS_CHECK_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
    const int ph = ctx->ev_phase[i] & 0xff;
    ctx->phase_ms[ph] += ms;
    ctx->phase_n[ph] += 1;
  }
  ctx->ev_used = 0;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_set_timing(seemps_ctx* ctx, int enabled) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  if (!enabled) SEEMPS_TRY(timing_flush(ctx));
  ctx->timing = enabled ? 1 : 0;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_get_timing(seemps_ctx* ctx, double* ms_out, long long* count_out,
                                           int reset) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_TRY(timing_flush(ctx));
  for (int i = 0; i < SEEMPS_PHASE_COUNT; ++i) {
    if (ms_out) ms_out[i] = ctx->phase_ms[i];
    if (count_out) count_out[i] = ctx->phase_n[i];
    if (reset) {
      ctx->phase_ms[i] = 0.0;
      ctx->phase_n[i] = 0;
    }
  }
  return SEEMPS_OK;
}

seemps_status copy_scalar_to_host(seemps_ctx* ctx, const void* dptr, void* hptr, size_t bytes) {
  SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(hptr, dptr, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_workspace_bytes(int chi_max, int d, int D_max, int krylov_dim,
                                                int chib_max, size_t* bytes_out) {
  if (!bytes_out || chi_max < 1 || d < 1 || D_max < 1 || krylov_dim < 1 || chib_max < 0)
    return SEEMPS_ERR_INVALID;
  size_t heff = heff_workspace_bytes(chi_max, d, D_max);
  size_t env = env_workspace_bytes(chi_max, d, D_max);
  size_t lz = lanczos_workspace_bytes(chi_max, d, D_max, krylov_dim);
  size_t pcg = pcg_workspace_bytes(chi_max, d, D_max);
  size_t svd = svd_workspace_bytes(chi_max * d, chi_max * d);
  size_t nloc = (size_t)chi_max * d * d * chi_max;
  // the sweep keeps theta, energies and a few scalars alongside the larger of
  // the local solver (which nests the matvec) and the split
  size_t solver = lz > pcg ? lz : pcg;
  size_t big = solver > svd ? solver : svd;
  if (env > big) big = env;
  // the MPO-MPS product: effective operator and environments between x
  // (bond chi_max) and b (bond chib_max), plus b's two-site tensor
  const int cm = chib_max > chi_max ? chib_max : chi_max;
  const size_t heff_b = heff_workspace_bytes(cm, d, D_max), env_b = env_workspace_bytes(cm, d, D_max);
  if (heff_b > big) big = heff_b;
  if (env_b > big) big = env_b;
  size_t lin = (size_t)chi_max * (chib_max > 0 ? chib_max : 1) * d * d * 8 * 4 + 4096 +
               (size_t)chib_max * chib_max * d * d * 8;
  size_t total = 512 + big + heff / 8 + nloc * 8 * 2 + lin + (size_t)64 * 256 + (1 << 20);
  *bytes_out = total;
  return SEEMPS_OK;
}

// ----------------------------------------------------------------- FP64 GEMM
// 64 x 64 output tile per 256-thread block, K staged 16 at a time in shared
// memory.  Each thread owns a 4 x 4 strided micro-tile (rows ty + 16 i,
// columns tx + 16 j) so that shared-memory reads are broadcasts (A) or
// consecutive doubles (B).  The global loads pick the thread order that
// makes the operand's unit-stride dimension the fast one.
namespace {
constexpr int DG_BM = 64, DG_BN = 64, DG_BK = 16;

__global__ void __launch_bounds__(256) dgemm_kernel(DgemmArgs a) {
  if (a.skip && *(volatile const int*)a.skip) return;
  __shared__ double As[DG_BK][DG_BM + 1];
  __shared__ double Bs[DG_BK][DG_BN + 1];
  const int b = blockIdx.z;
  const double* A = a.A + (ll)b * a.bsA;
  const double* B = a.B + (ll)b * a.bsB;
  double* C = a.C + (ll)b * a.bsC;
  const int m0 = blockIdx.y * DG_BM, n0 = blockIdx.x * DG_BN;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const bool a_kfast = (a.sAk == 1);
  const bool b_nfast = (a.sBn == 1) || (a.sBk != 1);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < a.K; k0 += DG_BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = t + 256 * q;
      int mm, kk;
      if (a_kfast) { kk = e & 15; mm = e >> 4; } else { mm = e & 63; kk = e >> 6; }
      int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < a.M && gk < a.K) ? A[(ll)gm * a.sAm + (ll)gk * a.sAk] : 0.0;
      int nn;
      if (b_nfast) { nn = e & 63; kk = e >> 6; } else { kk = e & 15; nn = e >> 4; }
      int gn = n0 + nn;
      gk = k0 + kk;
      Bs[kk][nn] = (gn < a.N && gk < a.K) ? B[(ll)gk * a.sBk + (ll)gn * a.sBn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DG_BK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= a.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= a.N) continue;
      double* c = C + (ll)gm * a.sCm + (ll)gn * a.sCn;
      double v = a.alpha * acc[i][j];
      if (a.beta != 0.0) v = fma(a.beta, *c, v);
      *c = v;
    }
  }
}
}  // namespace

seemps_status dgemm(seemps_ctx* ctx, const DgemmArgs& a) {
  if (a.M <= 0 || a.N <= 0 || a.batch <= 0) return SEEMPS_OK;
  if (a.K <= 0) {
    seemps_set_error(ctx, "dgemm: K = %d", a.K);
    return SEEMPS_ERR_INVALID;
  }
  dim3 grid(ceil_div(a.N, DG_BN), ceil_div(a.M, DG_BM), a.batch);
  if (grid.y > 65535 || grid.z > 65535) {
    seemps_set_error(ctx, "dgemm: grid too large (M=%d, batch=%d)", a.M, a.batch);
    return SEEMPS_ERR_INVALID;
  }
  DgemmArgs args = a;
  args.skip = ctx->skip;
  dgemm_kernel<<<grid, 256, 0, ctx->stream>>>(args);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}
