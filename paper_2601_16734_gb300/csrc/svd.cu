// Truncated SVD split of the two-site vector (Sect. 2.3): one-sided Jacobi
// (Hestenes) in FP64 (FP32 for the bf16x3 sweep), the truncation rank in
// FP64, and the re-layout of the kept factors into the new site tensors.
//
// The p = min(m, n) columns of X (X = M if n <= m, else X = M^T) are
// orthogonalised by plane rotations applied from the right; the same
// rotations accumulate in Q (p x p, starting at the identity).  Each column j
// of the stacked matrix G = [X; Q] is stored contiguously (length len + p,
// len = max(m, n)).  At convergence X = U S (columns orthogonal), so
// s_j = |X_j|, and M = U S Q^T (n <= m) or M = Q S U^T (n > m).
//
// Pairs follow the round-robin (circle) schedule: p' - 1 steps of p'/2
// disjoint pairs cover every pair once per sweep (p' = p rounded up to even).
// A pair is rotated when |x_a . x_b| > tol * |x_a| |x_b| with
// tol = max(1e-15, 2 sqrt(len) eps); a sweep without rotations ends the
// iteration.  Small problems (p <= 128) run every sweep inside one CTA (one
// warp per pair); larger ones run every sweep inside one cooperative launch
// (one CTA per pair, a bounded grid barrier between steps).
#include <math.h>

#include "common.cuh"
#include "timing.cuh"

namespace {

template <typename T> struct Eps;
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };

template <typename T>
__device__ __forceinline__ T block_sum_t(T v, T* sh);
template <>
__device__ __forceinline__ double block_sum_t<double>(double v, double* sh) { return block_sum(v, sh); }
template <>
__device__ __forceinline__ float block_sum_t<float>(float v, float* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_f(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  float t = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : 0.0f;
  if (w == 0) t = warp_sum_f(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  float r = sh[0];
  __syncthreads();
  return r;
}
__device__ __forceinline__ double wsum(double v) { return warp_sum(v); }
__device__ __forceinline__ float wsum(float v) { return warp_sum_f(v); }

// Grid-wide barrier for a cooperative launch, bounded: a block that waits
// longer than SEEMPS_WAIT_CLOCKS gives up and reports failure.
__device__ bool grid_barrier(unsigned* arrive, unsigned* gen, unsigned nblk) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = gen;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned prev = atomicAdd(arrive, 1u);
    if (prev == nblk - 1) {
      atomicExch(arrive, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > SEEMPS_WAIT_CLOCKS) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

__device__ __forceinline__ void rr_pair(int step, int k, int pp, int* a, int* b) {
  // circle method: player pp-1 fixed; the others rotate with the step
  if (k == 0) {
    *a = step;
    *b = pp - 1;
  } else {
    const int q = pp - 1;
    *a = (step + k) % q;
    *b = (step - k + q) % q;
  }
}

template <typename T>
__device__ __forceinline__ void jacobi_rotation(T alpha, T beta, T gamma, T* c, T* s) {
  const T zeta = (beta - alpha) / (T(2) * gamma);
  T t;
  if (fabs(zeta) > T(1e18)) {
    t = T(0.5) / zeta;
  } else {
    t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
  }
  *c = T(1) / sqrt(T(1) + t * t);
  *s = *c * t;
}

// G[j][i] = X(i, j) for i < len; Q part = identity.
template <typename T>
__global__ void svd_load_kernel(const double* __restrict__ M, int m, int n, int p, int len,
                                int transposed, T* __restrict__ G) {
  const ll colen = (ll)len + p;
  const ll total = colen * p;
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < total; e += (ll)gridDim.x * blockDim.x) {
    const int j = (int)(e / colen), i = (int)(e % colen);
    double v;
    if (i < len) {
      v = transposed ? M[(ll)j * n + i] : M[(ll)i * n + j];  // X = M^T : X(i, j) = M(j, i)
    } else {
      v = (i - len == j) ? 1.0 : 0.0;
    }
    G[e] = (T)v;
  }
}

// All sweeps in one cooperative launch.  A block of 1024 threads holds 8
// independent groups of 128 threads (4 warps); group g of block b handles
// pairs g + 8 b, g + 8 b + 8 grid, ... of every step.  A group reduces its
// three dot products with warp shuffles and one named barrier, so groups
// never wait on each other inside a step; blocks meet at a bounded grid
// barrier between steps.  Each block counts its rotations over a sweep and
// adds them to counts[sweep] once, before the sweep's last barrier; a sweep
// without rotations ends the iteration.
constexpr int GT = 128;   // threads per pair group
constexpr int GPB = 8;    // groups per block

__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(GT) : "memory");
}

template <typename T>
__global__ void __launch_bounds__(GT * GPB) svd_coop_kernel(T* __restrict__ G, int p, int pp, int len,
                                                            T tol, int max_sweeps,
                                                            int* __restrict__ counts, unsigned* bar,
                                                            int* sweeps_out, int* status) {
  __shared__ T red[GPB][4][3];
  __shared__ T rot[GPB][2];
  __shared__ int flag[GPB];
  __shared__ int block_rot;
  const int grp = threadIdx.x / GT, gt = threadIdx.x % GT, gw = gt >> 5, lane = gt & 31;
  const int ngroups = gridDim.x * GPB;
  const int gid = blockIdx.x * GPB + grp;
  const ll colen = (ll)len + p;
  const unsigned nblk = gridDim.x;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) block_rot = 0;
    __syncthreads();
    for (int step = 0; step < pp - 1; ++step) {
      for (int k = gid; k < pp / 2; k += ngroups) {
        int a, b;
        rr_pair(step, k, pp, &a, &b);
        if (a >= p || b >= p) continue;  // uniform within the group
        if (a > b) { int t = a; a = b; b = t; }
        T* xa = G + (ll)a * colen;
        T* xb = G + (ll)b * colen;
        // FP32 (or FP64) partial sums: 16 products per thread then a
        // 7-level tree, an error near 23 eps relative to sum |u v|, well
        // under the rotation threshold
        T saa = 0, sbb = 0, sab = 0;
#pragma unroll 4
        for (int i = gt; i < len; i += GT) {
          const T u = xa[i], v = xb[i];
          saa = fma(u, u, saa);
          sbb = fma(v, v, sbb);
          sab = fma(u, v, sab);
        }
        saa = wsum(saa);
        sbb = wsum(sbb);
        sab = wsum(sab);
        if (lane == 0) {
          red[grp][gw][0] = saa;
          red[grp][gw][1] = sbb;
          red[grp][gw][2] = sab;
        }
        group_sync(grp);
        if (gt == 0) {
          T A = 0, B = 0, C = 0;
          for (int w = 0; w < GT / 32; ++w) {
            A += red[grp][w][0];
            B += red[grp][w][1];
            C += red[grp][w][2];
          }
          const int doit = (C != T(0) && fabs(C) > tol * sqrt(A) * sqrt(B)) ? 1 : 0;
          flag[grp] = doit;
          if (doit) {
            T c, sn;
            jacobi_rotation<T>(A, B, C, &c, &sn);
            rot[grp][0] = c;
            rot[grp][1] = sn;
            atomicAdd(&block_rot, 1);
          }
        }
        group_sync(grp);
        if (flag[grp]) {
          const T c = rot[grp][0], sn = rot[grp][1];
          for (ll i = gt; i < colen; i += GT) {
            const T u = xa[i], v = xb[i];
            xa[i] = c * u - sn * v;
            xb[i] = sn * u + c * v;
          }
        }
        group_sync(grp);  // red/rot/flag are reused by the group's next pair
      }
      if (step == pp - 2) {
        __syncthreads();
        if (threadIdx.x == 0 && block_rot) atomicAdd(counts + sweep, block_rot);
      }
      if (!grid_barrier(bar, bar + 1, nblk)) {
        if (threadIdx.x == 0) post_status(status, SEEMPS_ERR_TIMEOUT);
        return;
      }
    }
    if (*(volatile int*)(counts + sweep) == 0) break;  // same value in every block after the barrier
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = sweep;
}

// All sweeps in one CTA of 1024 threads: warp w handles pairs w, w + 32, ...
// of each step.  Used for p <= 128.
template <typename T>
__global__ void __launch_bounds__(1024) svd_small_kernel(T* __restrict__ G, int p, int pp,
                                                         int len, T tol, int max_sweeps,
                                                         int* __restrict__ sweeps_out) {
  __shared__ int rotated;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const ll colen = (ll)len + p;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int step = 0; step < pp - 1; ++step) {
      for (int k = warp; k < pp / 2; k += 32) {
        int a, b;
        rr_pair(step, k, pp, &a, &b);
        if (a >= p || b >= p) continue;
        if (a > b) { int t = a; a = b; b = t; }
        T* xa = G + (ll)a * colen;
        T* xb = G + (ll)b * colen;
        T saa = 0, sbb = 0, sab = 0;
        for (int i = lane; i < len; i += 32) {
          const T u = xa[i], v = xb[i];
          saa = fma(u, u, saa);
          sbb = fma(v, v, sbb);
          sab = fma(u, v, sab);
        }
        saa = wsum(saa);
        sbb = wsum(sbb);
        sab = wsum(sab);
        if (sab != T(0) && fabs(sab) > tol * sqrt(saa) * sqrt(sbb)) {
          T c, s;
          jacobi_rotation<T>(saa, sbb, sab, &c, &s);
          for (ll i = lane; i < colen; i += 32) {
            const T u = xa[i], v = xb[i];
            xa[i] = c * u - s * v;
            xb[i] = s * u + c * v;
          }
          if (lane == 0) rotated = 1;
        }
        __syncwarp();
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  if (threadIdx.x == 0) *sweeps_out = sweep;
}

// s[j] = |X_j| (one block per column)
template <typename T>
__global__ void __launch_bounds__(256) svd_norms_kernel(const T* __restrict__ G, int p,
                                                        int len, double* __restrict__ s) {
  __shared__ double sh[32];
  const ll colen = (ll)len + p;
  const T* x = G + (ll)blockIdx.x * colen;
  double acc = 0.0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) acc = fma((double)x[i], (double)x[i], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) s[blockIdx.x] = sqrt(acc);
}

// perm[rank] = j with rank = #{i : s_i > s_j or (s_i == s_j and i < j)};
// sorted[rank] = s_j.  Descending, ties by column index.
__global__ void svd_sort_kernel(const double* __restrict__ s, int p, int* __restrict__ perm,
                                double* __restrict__ sorted) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x) {
    const double v = s[j];
    int r = 0;
    for (int i = 0; i < p; ++i) {
      const double u = s[i];
      r += (u > v || (u == v && i < j)) ? 1 : 0;
    }
    perm[r] = j;
    sorted[r] = v;
  }
}

// The truncation rule of Sect. 2.3, one thread, fixed summation order.
// out[0] = discarded fraction, out[1] = |S_r|; rank[0] = r.
__global__ void trunc_rank_kernel(const double* __restrict__ s, int n, int chi_max, double tol,
                                  int rule, int* __restrict__ rank, double* __restrict__ out) {
  if (threadIdx.x || blockIdx.x) return;
  int r;
  double total = 0.0;
  for (int j = n - 1; j >= 0; --j) total = __dadd_rn(total, __dmul_rn(s[j], s[j]));
  if (rule == SEEMPS_TRUNC_RELATIVE) {
    const double thr = __dmul_rn(tol, s[0]);
    r = 0;
    for (int j = 0; j < n; ++j)
      if (s[j] > thr) ++r;
  } else {
    const double limit = __dmul_rn(tol, total);
    r = n;
    double tail = 0.0;
    for (int j = n - 1; j >= 1; --j) {
      tail = __dadd_rn(tail, __dmul_rn(s[j], s[j]));
      if (tail <= limit) r = j;
      else break;
    }
  }
  if (r > chi_max) r = chi_max;
  if (r < 1) r = 1;
  double kept = 0.0, disc = 0.0;
  for (int j = n - 1; j >= r; --j) disc = __dadd_rn(disc, __dmul_rn(s[j], s[j]));
  for (int j = r - 1; j >= 0; --j) kept = __dadd_rn(kept, __dmul_rn(s[j], s[j]));
  rank[0] = r;
  if (out) {
    out[0] = total > 0.0 ? disc / total : 0.0;
    out[1] = sqrt(kept);
  }
}

// Output factors.  `xside_left`: the left factor comes from X (n <= m) or
// from Q (n > m).  Column j of the kept factors is column perm[j] of G.
// The factor on the X side is divided by s (it holds U S); the absorbing
// side is multiplied by sigma_j = s_j (or s_j / |S_r| when normalising).
template <typename T>
struct SplitOut {
  const T* G;
  const int* perm;
  const double* sorted;
  const int* rank;
  const double* aux;  // aux[1] = |S_r|
  int m, n, p, len;
  int xside_left;     // 1 if the left factor is built from X
  int absorb;         // SEEMPS_ABSORB_RIGHT / LEFT
  int normalize;
  double* A_left;     // m x r
  double* A_right;    // r x n
};

template <typename T>
__device__ __forceinline__ double col_factor(const SplitOut<T>& o, int j, bool left) {
  const double sj = o.sorted[j];
  const double sig = o.normalize ? sj / o.aux[1] : sj;
  const bool from_x = left ? (o.xside_left != 0) : (o.xside_left == 0);
  const bool absorbs = left ? (o.absorb == SEEMPS_ABSORB_LEFT) : (o.absorb == SEEMPS_ABSORB_RIGHT);
  double f = absorbs ? sig : 1.0;
  if (from_x) f = (sj > 0.0) ? f / sj : 0.0;
  return f;
}

// A_left[i][j] = f_j * G[perm j][row i of the left side], tiled transpose.
template <typename T>
__global__ void split_left_kernel(SplitOut<T> o) {
  __shared__ double tile[32][33];
  const int r = *o.rank;
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  if (j0 >= r) return;
  const ll colen = (ll)o.len + o.p;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int off = o.xside_left ? 0 : o.len;                 // X part or Q part of the column
  for (int jj = ty; jj < 32; jj += 8) {
    const int j = j0 + jj, i = i0 + tx;
    double v = 0.0;
    if (j < r && i < o.m) v = (double)o.G[(ll)o.perm[j] * colen + off + i] * col_factor(o, j, true);
    tile[jj][tx] = v;
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + tx;
    if (i < o.m && j < r) o.A_left[(ll)i * r + j] = tile[tx][ii];
  }
}

// A_right[j][c] = f_j * G[perm j][element c of the right side]
template <typename T>
__global__ void split_right_kernel(SplitOut<T> o) {
  const int r = *o.rank;
  const int j = blockIdx.y;
  if (j >= r) return;
  const ll colen = (ll)o.len + o.p;
  const int off = o.xside_left ? o.len : 0;
  const double f = col_factor(o, j, false);
  const T* src = o.G + (ll)o.perm[j] * colen + off;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < o.n; c += gridDim.x * blockDim.x)
    o.A_right[(ll)j * o.n + c] = (double)src[c] * f;
}

}  // namespace

size_t svd_workspace_bytes(int m, int n) {
  const size_t p = (size_t)(m < n ? m : n), len = (size_t)(m > n ? m : n);
  return (len + p) * p * 8 + p * 8 * 3 + p * 4 + 4096;
}

extern "C" seemps_status seemps_truncation_rank(seemps_ctx* ctx, int n, const double* s,
                                                const seemps_strategy* st, int* rank_out) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, s && st && rank_out && n > 0, "truncation_rank: bad argument");
  SEEMPS_REQUIRE(ctx, st->chi_max >= 1, "truncation_rank: chi_max < 1");
  trunc_rank_kernel<<<1, 32, 0, ctx->stream>>>(s, n, st->chi_max, st->tol, st->rule, rank_out, nullptr);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

template <typename T>
seemps_status svd_run(seemps_ctx* ctx, int m, int n, const double* theta, const seemps_strategy* st,
                      int absorb, int normalize, double* A_left, double* A_right, double* S,
                      int* rank_out, double* discarded_out, int max_sweeps) {
  const bool transposed = n > m;
  const int p = transposed ? m : n, len = transposed ? n : m;
  const int pp = p + (p & 1);
  T* G;
  double *s, *sorted, *aux;
  int *perm, *counters;
  unsigned* bar;
  SEEMPS_TRY(ws_alloc(ctx, ((size_t)len + p) * p, &G));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &s));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &sorted));
  SEEMPS_TRY(ws_alloc(ctx, 4, &aux));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &perm));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)max_sweeps + 2, &counters));
  SEEMPS_TRY(ws_alloc(ctx, 2, &bar));
  const T tol = (T)fmax(Eps<T>::v * 4.0, 2.0 * sqrt((double)len) * Eps<T>::v);
  svd_load_kernel<T><<<stride_grid(ctx, ((ll)len + p) * p, 256, 8), 256, 0, ctx->stream>>>(
      theta, m, n, p, len, transposed ? 1 : 0, G);
  SEEMPS_LAUNCHED(ctx);
  if (p > 1) {
    if (p <= 128) {
      svd_small_kernel<T><<<1, 1024, 0, ctx->stream>>>(G, p, pp, len, tol, max_sweeps, counters + max_sweeps);
      SEEMPS_LAUNCHED(ctx);
    } else {
      SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(counters, 0, sizeof(int) * (max_sweeps + 2), ctx->stream));
      SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(bar, 0, sizeof(unsigned) * 2, ctx->stream));
      int per_sm = 0;
      SEEMPS_CHECK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, svd_coop_kernel<T>,
                                                                           GT * GPB, 0));
      int blocks = per_sm * ctx->sm_count;
      const int want = ceil_div(pp / 2, GPB);
      if (blocks > want) blocks = want;
      if (blocks < 1) {
        seemps_set_error(ctx, "svd: cooperative kernel cannot be resident");
        return SEEMPS_ERR_UNSUPPORTED;
      }
      int* sweeps_out = counters + max_sweeps;
      int* status = ctx->d_status;
      T tolv = tol;
      void* args[] = {&G, (void*)&p, (void*)&pp, (void*)&len, &tolv, &max_sweeps, &counters, &bar,
                      &sweeps_out, &status};
      SEEMPS_CHECK_CUDA(ctx, cudaLaunchCooperativeKernel((void*)svd_coop_kernel<T>, dim3(blocks),
                                                         dim3(GT * GPB), args, 0, ctx->stream));
      SEEMPS_LAUNCHED(ctx);
    }
  }
  svd_norms_kernel<T><<<p, 256, 0, ctx->stream>>>(G, p, len, s);
  SEEMPS_LAUNCHED(ctx);
  svd_sort_kernel<<<ceil_div(p, 256), 256, 0, ctx->stream>>>(s, p, perm, sorted);
  SEEMPS_LAUNCHED(ctx);
  trunc_rank_kernel<<<1, 32, 0, ctx->stream>>>(sorted, p, st->chi_max, st->tol, st->rule, rank_out, aux);
  SEEMPS_LAUNCHED(ctx);
  if (discarded_out)
    SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(discarded_out, aux, sizeof(double), cudaMemcpyDeviceToDevice,
                                           ctx->stream));
  if (S)
    SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(S, sorted, sizeof(double) * p, cudaMemcpyDeviceToDevice,
                                           ctx->stream));
  SplitOut<T> o;
  o.G = G;
  o.perm = perm;
  o.sorted = sorted;
  o.rank = rank_out;
  o.aux = aux;
  o.m = m;
  o.n = n;
  o.p = p;
  o.len = len;
  o.xside_left = transposed ? 0 : 1;
  o.absorb = absorb;
  o.normalize = normalize;
  o.A_left = A_left;
  o.A_right = A_right;
  const int rmax = p < st->chi_max ? p : st->chi_max;
  dim3 gl(ceil_div(m, 32), ceil_div(rmax, 32));
  split_left_kernel<T><<<gl, 256, 0, ctx->stream>>>(o);
  SEEMPS_LAUNCHED(ctx);
  dim3 gr(ceil_div(n, 256) < 8 ? ceil_div(n, 256) : 8, rmax);
  split_right_kernel<T><<<gr, 256, 0, ctx->stream>>>(o);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_svd_truncate(seemps_ctx* ctx, int m, int n, const double* theta,
                                             const seemps_strategy* st, int absorb, int normalize,
                                             double* A_left, double* A_right, double* S,
                                             int* rank_out, double* discarded_out,
                                             int max_sweeps, int precision) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, theta && st && A_left && A_right && rank_out, "svd_truncate: null argument");
  SEEMPS_REQUIRE(ctx, m > 0 && n > 0, "svd_truncate: empty matrix %d x %d", m, n);
  SEEMPS_REQUIRE(ctx, st->chi_max >= 1, "svd_truncate: chi_max < 1");
  SEEMPS_REQUIRE(ctx, absorb == SEEMPS_ABSORB_RIGHT || absorb == SEEMPS_ABSORB_LEFT,
                 "svd_truncate: bad absorb");
  SEEMPS_REQUIRE(ctx, precision == SEEMPS_FP64 || precision == SEEMPS_BF16X3,
                 "svd_truncate: unknown precision");
  if (max_sweeps <= 0) max_sweeps = 40;
  WsFrame frame(ctx);
  PhaseTimer timer(ctx, SEEMPS_PHASE_SVD);
  if (precision == SEEMPS_FP64)
    return svd_run<double>(ctx, m, n, theta, st, absorb, normalize, A_left, A_right, S, rank_out,
                           discarded_out, max_sweeps);
  return svd_run<float>(ctx, m, n, theta, st, absorb, normalize, A_left, A_right, S, rank_out,
                        discarded_out, max_sweeps);
}
