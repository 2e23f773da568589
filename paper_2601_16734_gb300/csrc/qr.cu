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
constexpr int QT_NT = 128;            // trailing-update threads (row chunks)
constexpr int QT_CPW = 4;             // trailing columns per CTA

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
                                              float* diag, float (*G)[W], float (*Rtop)[W], int i0, int M, int j0,
                                              int wn, int tid, int lane, int warp) {
  constexpr int j = J;
  tau[j] = 0.f;
  if (j >= wn) return;  // uniform
  const int dr = j0 + j;  // row of the diagonal entry
  // rows j0 .. dr - 1 of column j are final entries of R: keep them aside
  // and zero them, so that p[j] below holds v_j with no row tests
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    if (i < dr) {
      Rtop[i - j0][j] = p[j][r];
      p[j][r] = 0.f;
    }
  }
  float x2[2] = {0.f, 0.f};
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    if (i == dr) x2[1] = p[j][r];
    else x2[0] = fmaf(p[j][r], p[j][r], x2[0]);
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
  for (int r = 0; r < R; ++r) p[j][r] = (i0 + r == dr) ? 1.f : p[j][r] * sc;
  if (i0 <= dr && dr < i0 + R) diag[j] = beta;
  if (tj != 0.f) {
    // one reduction: d_c = v_j . p_c for the later panel columns c > j (to
    // apply H_j = I - tau v v^T) and G(a, j) = v_a . v_j for the earlier
    // reflectors a < j (for T); v_j vanishes outside rows dr .. M - 1
    float d[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      float acc = 0.f;
      if (c != j && c < W) {
#pragma unroll
        for (int r = 0; r < R; ++r) acc = fmaf(p[j][r], p[c][r], acc);
      }
      d[c] = acc;
    }
    qr_cta_sum<16>(d, red, tot, lane, warp);
    if (tid < j) G[tid][j] = tot[tid];
#pragma unroll
    for (int c = j + 1; c < W; ++c) {
      const float f = tj * tot[c];
#pragma unroll
      for (int r = 0; r < R; ++r) p[c][r] = fmaf(-f, p[j][r], p[c][r]);
    }
  }
}

template <int R, int W, int... J>
__device__ __forceinline__ void qr_panel_steps(std::integer_sequence<int, J...>, float (&p)[W][R], float (&tau)[W],
                                               float (*red)[16], float* tot, float* diag, float (*G)[W],
                                               float (*Rtop)[W], int i0, int M, int j0, int wn, int tid, int lane,
                                               int warp) {
  (qr_panel_step<R, W, J>(p, tau, red, tot, diag, G, Rtop, i0, M, j0, wn, tid, lane, warp), ...);
}

// Factor panel columns j0 .. j0 + wn - 1 (wn <= W) of the column-major
// M x N matrix A (leading dimension lda), rows j0 .. M - 1.  Thread t owns
// rows j0 + R t .. j0 + R t + R - 1.  On exit the panel holds R (diagonal and
// above) and the reflectors v_j (below the diagonal, v_j(j0 + j) = 1
// implied); T (W x W, row-major, upper triangular) is the compact-WY factor.
template <int R, int W>
__global__ void __launch_bounds__(QP_NT, 1) qr_panel_kernel(float* __restrict__ A, int lda, int M, int j0,
                                                            int wn, float* __restrict__ T,
                                                            float* __restrict__ Vt) {
  static_assert(W <= 16 && (W & (W - 1)) == 0 && R % 4 == 0, "panel shape");
  __shared__ float red[QP_NW][16];
  __shared__ float tot[16];
  __shared__ float diag[W];
  __shared__ float G[W][W];     // G(a, b) = v_a . v_b, a < b
  __shared__ float Rtop[W][W];  // R(j0 + i, j0 + j) for i < j
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = j0 + R * tid;
  const bool vec = (lda % 4 == 0) && (j0 % 4 == 0);
  float p[W][R];
#pragma unroll
  for (int c = 0; c < W; ++c) {
    const float* col = A + (ll)(j0 + c) * lda;
    if (c < wn && vec && i0 + R <= M) {
#pragma unroll
      for (int r = 0; r < R; r += 4) {
        const float4 q4 = *reinterpret_cast<const float4*>(col + i0 + r);
        p[c][r] = q4.x;
        p[c][r + 1] = q4.y;
        p[c][r + 2] = q4.z;
        p[c][r + 3] = q4.w;
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) p[c][r] = (c < wn && i0 + r < M) ? col[i0 + r] : 0.f;
    }
  }
  if (tid < W * W) G[tid / W][tid % W] = 0.f;  // ordered by the first reduction's barriers
  float tau[W];
  qr_panel_steps<R, W>(std::make_integer_sequence<int, W>{}, p, tau, red, tot, diag, G, Rtop, i0, M, j0, wn, tid,
                       lane, warp);
  __syncthreads();  // diag[] and G complete
#pragma unroll
  for (int c = 0; c < W; ++c) {
    if (c >= wn) break;
    float out[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + r;
      out[r] = i < j0 + c ? Rtop[i - j0][c] : (i == j0 + c ? diag[c] : p[c][r]);
    }
    float* col = A + (ll)(j0 + c) * lda;
    if (vec && i0 + R <= M) {
#pragma unroll
      for (int r = 0; r < R; r += 4)
        *reinterpret_cast<float4*>(col + i0 + r) = make_float4(out[r], out[r + 1], out[r + 2], out[r + 3]);
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (i0 + r < M) col[i0 + r] = out[r];
    }
  }
  // the reflectors row by row for the trailing update: Vt[ii][j] = v_j(j0 + ii),
  // zero above the diagonal, one on it
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    if (i >= M) break;
    float vr[W];
#pragma unroll
    for (int c = 0; c < W; ++c) vr[c] = c < wn ? p[c][r] : 0.f;
    float4* dst = reinterpret_cast<float4*>(Vt + (ll)(i - j0) * W);
#pragma unroll
    for (int c = 0; c < W; c += 4) dst[c / 4] = make_float4(vr[c], vr[c + 1], vr[c + 2], vr[c + 3]);
  }
  if (warp == 0) {
    // T(i, i) = tau_i;  T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i), column by
    // column; lane a keeps row a of T in registers
    float tr[W];
#pragma unroll
    for (int c = 0; c < W; ++c) tr[c] = 0.f;
#pragma unroll
    for (int c = 0; c < W; ++c)
      if (lane == c) tr[c] = tau[c];
#pragma unroll
    for (int i = 1; i < W; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < i; ++c) acc = fmaf(tr[c], G[c][i], acc);  // tr[c] = 0 for c < lane
      if (lane < i) tr[i] = -tau[i] * acc;
    }
    if (lane < W) {
#pragma unroll
      for (int c = 0; c < W; ++c) T[lane * W + c] = tr[c];
    }
  }
}

// A(:, c) <- (I - V T^T V^T) A(:, c) for trailing columns c >= c0, rows >= j0.
// A CTA updates QT_CPW columns; its QT_NT / 32 warps split the rows into
// chunks (partial V^T a reduced through shared memory), lanes stride over
// the rows of a chunk two rows at a time, and every element of V (row-major
// Vt, read through L1: it is the same for all CTAs) feeds QT_CPW FMAs.
template <int W>
__global__ void __launch_bounds__(QT_NT) qr_trail_kernel(float* __restrict__ A, int lda, int M, int N, int j0,
                                                         int c0, const float* __restrict__ T,
                                                         const float* __restrict__ Vt) {
  constexpr int NWARP = QT_NT / 32;
  __shared__ float Ts[W][W];
  __shared__ float wsum[NWARP][QT_CPW][W];
  __shared__ float ys[QT_CPW][W];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < W * W; e += QT_NT) Ts[e / W][e % W] = T[e];
  const int rows = M - j0;
  const int chunk = ((rows + NWARP - 1) / NWARP + 63) & ~63;
  const int rb = warp * chunk, re = min(rows, rb + chunk);
  const int cb = c0 + blockIdx.x * QT_CPW;
  float* a[QT_CPW];
  bool on[QT_CPW];
#pragma unroll
  for (int q = 0; q < QT_CPW; ++q) {
    on[q] = cb + q < N;
    a[q] = A + (ll)(on[q] ? cb + q : cb) * lda + j0;
  }
  auto vrow = [&](int ii, float (&v)[W]) {
    const float4* src = reinterpret_cast<const float4*>(Vt + (ll)ii * W);
#pragma unroll
    for (int c = 0; c < W; c += 4) {
      const float4 q4 = __ldg(src + c / 4);
      v[c] = q4.x;
      v[c + 1] = q4.y;
      v[c + 2] = q4.z;
      v[c + 3] = q4.w;
    }
  };
  float w[QT_CPW][W];
#pragma unroll
  for (int q = 0; q < QT_CPW; ++q)
#pragma unroll
    for (int j = 0; j < W; ++j) w[q][j] = 0.f;
  for (int ii = rb + lane; ii < re; ii += 64) {
    const int i2 = ii + 32;
    const bool two = i2 < re;
    float av[QT_CPW], bv[QT_CPW], v1[W], v2[W];
#pragma unroll
    for (int q = 0; q < QT_CPW; ++q) {
      av[q] = a[q][ii];
      bv[q] = two ? a[q][i2] : 0.f;
    }
    vrow(ii, v1);
    if (two) vrow(i2, v2);
    else {
#pragma unroll
      for (int j = 0; j < W; ++j) v2[j] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < W; ++j)
#pragma unroll
      for (int q = 0; q < QT_CPW; ++q) w[q][j] = fmaf(v2[j], bv[q], fmaf(v1[j], av[q], w[q][j]));
  }
#pragma unroll
  for (int q = 0; q < QT_CPW; ++q) {
    const float wt = rs_reduce<W>(w[q], lane);
    if (lane < W) wsum[warp][q][rs_index<W>(lane)] = wt;
  }
  __syncthreads();
  // y_q = T^T (V^T a_q): thread (q, b) computes entry b of column q
  if (tid < QT_CPW * W) {
    const int q = tid / W, bcol = tid % W;
    float yb = 0.f;
    for (int aa = 0; aa <= bcol; ++aa) {
      float wa = 0.f;
#pragma unroll
      for (int k = 0; k < NWARP; ++k) wa += wsum[k][q][aa];
      yb = fmaf(Ts[aa][bcol], wa, yb);
    }
    ys[q][bcol] = yb;
  }
  __syncthreads();
  float y[QT_CPW][W];
#pragma unroll
  for (int q = 0; q < QT_CPW; ++q)
#pragma unroll
    for (int j = 0; j < W; ++j) y[q][j] = ys[q][j];
  for (int ii = rb + lane; ii < re; ii += 64) {
    const int i2 = ii + 32;
    const bool two = i2 < re;
    float av[QT_CPW], bv[QT_CPW], v1[W], v2[W];
#pragma unroll
    for (int q = 0; q < QT_CPW; ++q) {
      av[q] = a[q][ii];
      bv[q] = two ? a[q][i2] : 0.f;
    }
    vrow(ii, v1);
    if (two) vrow(i2, v2);
    else {
#pragma unroll
      for (int j = 0; j < W; ++j) v2[j] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < W; ++j)
#pragma unroll
      for (int q = 0; q < QT_CPW; ++q) {
        av[q] = fmaf(-v1[j], y[q][j], av[q]);
        bv[q] = fmaf(-v2[j], y[q][j], bv[q]);
      }
#pragma unroll
    for (int q = 0; q < QT_CPW; ++q)
      if (on[q]) {
        a[q][ii] = av[q];
        if (two) a[q][i2] = bv[q];
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
seemps_status qr_run(seemps_ctx* ctx, float* A, int M, int N, float* Tbuf, float* Vt) {
  const int k = M < N ? M : N;
  for (int j0 = 0; j0 < k; j0 += W) {
    const int wn = (k - j0) < W ? (k - j0) : W;
    qr_panel_kernel<R, W><<<1, QP_NT, 0, ctx->stream>>>(A, M, M, j0, wn, Tbuf, Vt);
    SEEMPS_LAUNCHED(ctx);
    const int c0 = j0 + wn;
    if (c0 < N) {
      qr_trail_kernel<W><<<ceil_div(N - c0, QT_CPW), QT_NT, 0, ctx->stream>>>(A, M, M, N, j0, c0, Tbuf, Vt);
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
  float *Tbuf, *Vt;
  SEEMPS_TRY(ws_alloc(ctx, 256, &Tbuf));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)16 * M, &Vt));  // the panel's reflectors, row-major
  if (M <= 4 * QP_NT) SEEMPS_TRY((qr_run<4, 16>(ctx, A, M, N, Tbuf, Vt)));
  else SEEMPS_TRY((qr_run<8, 8>(ctx, A, M, N, Tbuf, Vt)));
  const int k = M < N ? M : N;
  dim3 grid(ceil_div(N, 32), ceil_div(k, 32));
  qr_rt_kernel<<<grid, 256, 0, ctx->stream>>>(A, M, k, N, X);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}
