// FP32 Householder QR, R factor only, used to precondition the one-sided
// Jacobi SVD of the mixed-precision sweep (Sect. 2.3 asks for a truncated
// SVD; how it is computed is an implementation choice).  For A = Q R the
// matrix R^T has the singular values of A and, as left singular vectors, the
// right singular vectors of A, so one-sided Jacobi on the columns of R^T
// yields the isometric factor directly; on R^T it needs far fewer sweeps than
// on A itself (the triangular factor is much closer to having orthogonal
// columns).
//
// Blocked right-looking Householder with panels of W columns: one CTA
// factors a panel held in registers (rows distributed over threads), forms
// the compact-WY factor T (H_0 ... H_{W-1} = I - V T V^T) and writes the
// reflectors below the diagonal; then a grid of CTAs applies
// Q^T = I - V T^T V^T to the trailing columns (V staged in shared memory, one
// warp per column, lanes striding over rows).
#include <utility>

#include "common.cuh"

namespace {

constexpr int QP_NT = 512;            // panel kernel threads
constexpr int QP_NW = QP_NT / 32;
constexpr int QT_NT = 256;            // trailing-update threads
constexpr int QT_COLS = 16;           // trailing columns per CTA (two per warp)

// CTA-wide sums of NV values (NV <= 16, a power of two): every thread reads
// the totals from tot[] after the call.
template <int NV>
__device__ __forceinline__ void qr_cta_sum(float (&x)[NV], float (*red)[16], float* tot, int lane, int warp) {
  const float t = rs_reduce<NV>(x, lane);
  if (lane < NV) red[warp][rs_index<NV>(lane)] = t;
  __syncthreads();
  if (warp == 0 && lane < NV) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < QP_NW; ++w) s += red[w][lane];
    tot[lane] = s;
  }
  __syncthreads();
}

// One Householder step of the panel factorization (column J of the panel).
template <int R, int W, int J>
__device__ __forceinline__ void qr_panel_step(float (&p)[W][R], float (&tau)[W], float (*red)[16], float* tot,
                                              float* diag, float (*G)[W], int i0, int M, int j0, int wn,
                                              int tid, int lane, int warp) {
  constexpr int j = J;
  tau[j] = 0.f;
  if (j >= wn) return;  // uniform
  const int dr = j0 + j;  // row of the diagonal entry
  float x2[2] = {0.f, 0.f};
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    if (i > dr && i < M) x2[0] = fmaf(p[j][r], p[j][r], x2[0]);
    if (i == dr) x2[1] = p[j][r];
  }
  qr_cta_sum<2>(x2, red, tot, lane, warp);
  const float s2 = tot[0], x0 = tot[1];
  float beta = x0, tj = 0.f, sc = 0.f;
  if (s2 > 0.f) {
    const float nrm = sqrtf(fmaf(x0, x0, s2));
    beta = x0 >= 0.f ? -nrm : nrm;
    tj = (beta - x0) / beta;
    sc = 1.f / (x0 - beta);
  }
  tau[j] = tj;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    if (i > dr && i < M) p[j][r] *= sc;
    else if (i == dr) p[j][r] = 1.f;
  }
  if (i0 <= dr && dr < i0 + R) diag[j] = beta;
  if (tj != 0.f) {
    // one reduction: d_c = v_j . p_c for the later panel columns c > j
    // (to apply H_j = I - tau v v^T) and G(a, j) = v_a . v_j for the
    // earlier reflectors a < j (for T); all over rows >= dr, where v_j lives
    float d[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      float acc = 0.f;
      if (c != j && c < W) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int i = i0 + r;
          if (i >= dr && i < M) acc = fmaf(p[j][r], p[c][r], acc);
        }
      }
      d[c] = acc;
    }
    qr_cta_sum<16>(d, red, tot, lane, warp);
    if (tid < j) G[tid][j] = tot[tid];
#pragma unroll
    for (int c = j + 1; c < W; ++c) {
      const float f = tj * tot[c];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = i0 + r;
        if (i >= dr && i < M) p[c][r] = fmaf(-f, p[j][r], p[c][r]);
      }
    }
  }
}

template <int R, int W, int... J>
__device__ __forceinline__ void qr_panel_steps(std::integer_sequence<int, J...>, float (&p)[W][R], float (&tau)[W],
                                               float (*red)[16], float* tot, float* diag, float (*G)[W], int i0,
                                               int M, int j0, int wn, int tid, int lane, int warp) {
  (qr_panel_step<R, W, J>(p, tau, red, tot, diag, G, i0, M, j0, wn, tid, lane, warp), ...);
}

// Factor panel columns j0 .. j0 + wn - 1 (wn <= W) of the column-major
// M x N matrix A (leading dimension lda), rows j0 .. M - 1.  Thread t owns
// rows R t .. R t + R - 1.  On exit the panel holds R (diagonal and above)
// and the reflectors v_j (below the diagonal, v_j(j0 + j) = 1 implied);
// T (W x W, row-major, upper triangular) is the compact-WY factor.
template <int R, int W>
__global__ void __launch_bounds__(QP_NT, 1) qr_panel_kernel(float* __restrict__ A, int lda, int M, int j0,
                                                            int wn, float* __restrict__ T) {
  static_assert(W <= 16 && (W & (W - 1)) == 0, "panel width");
  __shared__ float red[QP_NW][16];
  __shared__ float tot[16];
  __shared__ float diag[W];
  __shared__ float G[W][W];   // G(a, b) = v_a . v_b, a < b
  __shared__ float Ts[W][W];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = R * tid;
  float p[W][R];
#pragma unroll
  for (int c = 0; c < W; ++c)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + r;
      p[c][r] = (c < wn && i >= j0 && i < M) ? A[(ll)(j0 + c) * lda + i] : 0.f;
    }
  float tau[W];
  qr_panel_steps<R, W>(std::make_integer_sequence<int, W>{}, p, tau, red, tot, diag, G, i0, M, j0, wn, tid, lane,
                       warp);
  __syncthreads();  // diag[] complete
#pragma unroll
  for (int c = 0; c < W; ++c)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + r;
      if (c < wn && i >= j0 && i < M) A[(ll)(j0 + c) * lda + i] = (i == j0 + c) ? diag[c] : p[c][r];
    }
#pragma unroll
  for (int j = 0; j < W; ++j)
    if (tid == j) Ts[j][j] = tau[j];
  __syncthreads();
  if (warp == 0) {
    // T(i, i) = tau_i;  T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i), column by column
    for (int i = 1; i < W; ++i) {
      float acc = 0.f;
      if (lane < i)
        for (int c = lane; c < i; ++c) acc = fmaf(Ts[lane][c], G[c][i], acc);
      const float ti = Ts[i][i];
      __syncwarp();
      if (lane < i) Ts[lane][i] = -ti * acc;
      __syncwarp();
    }
    for (int e = lane; e < W * W; e += 32) {
      const int aa = e / W, bb = e % W;
      T[e] = aa <= bb ? Ts[aa][bb] : 0.f;
    }
  }
}

// A(:, c) <- (I - V T^T V^T) A(:, c) for trailing columns c >= c0, rows >= j0.
template <int W>
__global__ void __launch_bounds__(QT_NT) qr_trail_kernel(float* __restrict__ A, int lda, int M, int N, int j0,
                                                         int wn, int c0, const float* __restrict__ T) {
  extern __shared__ __align__(16) float qr_smem[];
  const int rows = M - j0;
  float* sv = qr_smem;               // [W][rows]: v_j restricted to rows >= j0
  __shared__ float Ts[W][W];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < W * rows; e += QT_NT) {
    const int j = e / rows, ii = e % rows, i = j0 + ii;
    float v = 0.f;
    if (j < wn) {
      if (i > j0 + j) v = A[(ll)(j0 + j) * lda + i];
      else if (i == j0 + j) v = 1.f;
    }
    sv[e] = v;
  }
  for (int e = tid; e < W * W; e += QT_NT) Ts[e / W][e % W] = T[e];
  __syncthreads();
#pragma unroll 1
  for (int q = 0; q < QT_COLS / (QT_NT / 32); ++q) {
    const int c = c0 + blockIdx.x * QT_COLS + q * (QT_NT / 32) + warp;
    if (c >= N) continue;  // warp-uniform
    float* a = A + (ll)c * lda + j0;
    float w[W];
#pragma unroll
    for (int j = 0; j < W; ++j) w[j] = 0.f;
    for (int ii = lane; ii < rows; ii += 32) {
      const float av = a[ii];
#pragma unroll
      for (int j = 0; j < W; ++j) w[j] = fmaf(sv[j * rows + ii], av, w[j]);
    }
    // warp totals: lane holds W-vector entry rs_index(lane)
    const float wt = rs_reduce<W>(w, lane);
    // y_b = sum_{a <= b} T(a, b) w_a ; lane b computes y_b
    float y = 0.f;
#pragma unroll
    for (int aa = 0; aa < W; ++aa) {
      // the lane holding w_aa: the lowest lane whose rs_index equals aa
      int src = 0;
#pragma unroll
      for (int m = 1, h = W / 2; h >= 1; m <<= 1, h >>= 1)
        if (aa & h) src |= m;
      const float wa = __shfl_sync(0xffffffffu, wt, src);
      if (lane < W && aa <= lane) y = fmaf(Ts[aa][lane], wa, y);
    }
    float yv[W];
#pragma unroll
    for (int j = 0; j < W; ++j) yv[j] = __shfl_sync(0xffffffffu, y, j);
    for (int ii = lane; ii < rows; ii += 32) {
      float av = a[ii];
#pragma unroll
      for (int j = 0; j < W; ++j) av = fmaf(-sv[j * rows + ii], yv[j], av);
      a[ii] = av;
    }
  }
}

// X[j][c] = R(j, c) for c >= j, 0 below: the transpose of the upper
// trapezoid of the factored A (k rows of R, N columns).
__global__ void qr_rt_kernel(const float* __restrict__ A, int lda, int k, int N, float* __restrict__ X) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int cc = ty; cc < 32; cc += 8) {
    const int c = c0 + cc, j = j0 + tx;
    tile[cc][tx] = (c < N && j < k && c >= j) ? A[(ll)c * lda + j] : 0.f;
  }
  __syncthreads();
  for (int jj = ty; jj < 32; jj += 8) {
    const int j = j0 + jj, c = c0 + tx;
    if (j < k && c < N) X[(ll)j * N + c] = tile[tx][jj];
  }
}

template <int R, int W>
seemps_status qr_run(seemps_ctx* ctx, float* A, int M, int N, float* Tbuf) {
  const int k = M < N ? M : N;
  const size_t smem_max = (size_t)W * M * sizeof(float);
  if (smem_max > 48 * 1024)
    SEEMPS_CHECK_CUDA(ctx, cudaFuncSetAttribute(qr_trail_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem_max));
  for (int j0 = 0; j0 < k; j0 += W) {
    const int wn = (k - j0) < W ? (k - j0) : W;
    qr_panel_kernel<R, W><<<1, QP_NT, 0, ctx->stream>>>(A, M, M, j0, wn, Tbuf);
    SEEMPS_LAUNCHED(ctx);
    const int c0 = j0 + wn;
    if (c0 < N) {
      const size_t smem = (size_t)W * (M - j0) * sizeof(float);
      qr_trail_kernel<W><<<ceil_div(N - c0, QT_COLS), QT_NT, smem, ctx->stream>>>(A, M, M, N, j0, wn, c0, Tbuf);
      SEEMPS_LAUNCHED(ctx);
    }
  }
  return SEEMPS_OK;
}

}  // namespace

bool qr_supported(int M, int N) { return M >= 1 && N >= 1 && M <= 4 * QP_NT * 2; }

seemps_status qr_r_transpose(seemps_ctx* ctx, float* A, int M, int N, float* X) {
  if (!qr_supported(M, N)) {
    seemps_set_error(ctx, "qr: %d rows exceed the panel kernel", M);
    return SEEMPS_ERR_UNSUPPORTED;
  }
  float* Tbuf;
  SEEMPS_TRY(ws_alloc(ctx, 256, &Tbuf));
  if (M <= 2 * QP_NT) SEEMPS_TRY((qr_run<2, 16>(ctx, A, M, N, Tbuf)));
  else if (M <= 4 * QP_NT) SEEMPS_TRY((qr_run<4, 16>(ctx, A, M, N, Tbuf)));
  else SEEMPS_TRY((qr_run<8, 8>(ctx, A, M, N, Tbuf)));
  const int k = M < N ? M : N;
  dim3 grid(ceil_div(N, 32), ceil_div(k, 32));
  qr_rt_kernel<<<grid, 256, 0, ctx->stream>>>(A, M, k, N, X);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}
