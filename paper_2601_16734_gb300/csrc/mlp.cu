// Learned local preconditioner for the PCG solve of the sweep.
//
// Per-entry features of the local system on the pair (i, i+1) of an N-site
// chain, entry j = (a, s, t, c):
//   x0 = log10(diag_j)/10, x1 = i/N, x2 = (i+1)/N, x3 = log10|L[a,:,a]|/10,
//   x4 = log10|R[c,:,c]|/10, x5 = s/(d-1), x6 = t/(d-1)
// -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> o = W3 h2 + b3 (7 -> 64 -> 64 -> 5)
// -> p_j = softplus(o0_j)/diag_j, U_jk = o_{1+k,j}/sqrt(n)  (k < 4)
// and the preconditioner z = P r = p * r + U (U^T r), symmetric positive
// definite by construction.  Training minimises |x* - P b|_A^2 / (x*^T b)
// over (local system, exact local solution) pairs with Adam.  Network
// arithmetic is FP32; p, U and the preconditioner apply are FP64.
//
// The backward pass recomputes the forward pass per entry, stores the layer
// activations and their gradients, and reduces the weight gradients with one
// thread per weight over all entries in a fixed order (deterministic).
#include <math.h>

#include "contract.cuh"

namespace {

constexpr int H = 64;        // hidden width
constexpr int F = 7;         // features
constexpr int NO = 5;        // outputs
constexpr int RK = 4;        // rank of the low-rank part
constexpr int NP = H * F + H + H * H + H + NO * H + NO;
constexpr int OW1 = 0, OB1 = OW1 + H * F, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + NO * H;
constexpr int MT = 128;      // threads of the per-entry kernels

__device__ __forceinline__ float softplus_f(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid_f(float x) { return 1.f / (1.f + expf(-x)); }

__device__ __forceinline__ bool stopped(const int* f) { return f && *(volatile const int*)f; }

// features X[j][0..6]
__global__ void features_kernel(const double* __restrict__ diag, const double* __restrict__ L,
                                const double* __restrict__ R, int chil, int chir, int d, int Dl,
                                int Dr, int site, int nsites, float* __restrict__ X) {
  const ll n = (ll)chil * d * d * chir;
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x) {
    const int c = (int)(e % chir);
    const int t = (int)((e / chir) % d);
    const int s = (int)((e / ((ll)chir * d)) % d);
    const int a = (int)(e / ((ll)chir * d * d));
    double ln = 0.0, rn = 0.0;
    for (int b = 0; b < Dl; ++b) {
      const double v = L[((ll)a * Dl + b) * chil + a];
      ln += v * v;
    }
    for (int f = 0; f < Dr; ++f) {
      const double v = R[((ll)c * Dr + f) * chir + c];
      rn += v * v;
    }
    float* x = X + e * F;
    x[0] = (float)(log10(diag[e]) / 10.0);
    x[1] = (float)site / (float)nsites;
    x[2] = (float)(site + 1) / (float)nsites;
    x[3] = (float)(log10(sqrt(ln) + 1e-300) / 10.0);
    x[4] = (float)(log10(sqrt(rn) + 1e-300) / 10.0);
    x[5] = d > 1 ? (float)s / (float)(d - 1) : 0.f;
    x[6] = d > 1 ? (float)t / (float)(d - 1) : 0.f;
  }
}

__device__ __forceinline__ void load_params(const float* __restrict__ P, float* sP) {
  for (int i = threadIdx.x; i < NP; i += blockDim.x) sP[i] = P[i];
  __syncthreads();
}

// forward for one entry; h1, h2 in registers
__device__ __forceinline__ void forward_entry(const float* sP, const float* x, float (&h1)[H],
                                              float (&h2)[H], float (&o)[NO]) {
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float acc = sP[OB1 + i];
#pragma unroll
    for (int k = 0; k < F; ++k) acc = fmaf(sP[OW1 + i * F + k], x[k], acc);
    h1[i] = tanhf(acc);
  }
#pragma unroll
  for (int j = 0; j < NO; ++j) o[j] = sP[OB3 + j];
#pragma unroll 4
  for (int i = 0; i < H; ++i) {
    float acc = sP[OB2 + i];
#pragma unroll
    for (int k = 0; k < H; ++k) acc = fmaf(sP[OW2 + i * H + k], h1[k], acc);
    h2[i] = tanhf(acc);
#pragma unroll
    for (int j = 0; j < NO; ++j) o[j] = fmaf(sP[OW3 + j * H + i], h2[i], o[j]);
  }
}

// p_j, U_j from the network (also keeps o for the backward pass)
__global__ void __launch_bounds__(MT) forward_kernel(const float* __restrict__ params,
                                                     const float* __restrict__ X,
                                                     const double* __restrict__ diag, ll n,
                                                     double* __restrict__ p, double* __restrict__ U,
                                                     float* __restrict__ O) {
  __shared__ float sP[NP];
  load_params(params, sP);
  const double inv_sqrt_n = 1.0 / sqrt((double)n);
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x) {
    float x[F];
#pragma unroll
    for (int k = 0; k < F; ++k) x[k] = X[e * F + k];
    float h1[H], h2[H], o[NO];
    forward_entry(sP, x, h1, h2, o);
    p[e] = (double)softplus_f(o[0]) / diag[e];
#pragma unroll
    for (int k = 0; k < RK; ++k) U[e * RK + k] = (double)o[1 + k] * inv_sqrt_n;
    if (O) {
#pragma unroll
      for (int j = 0; j < NO; ++j) O[e * NO + j] = o[j];
    }
  }
}

// partial[blk][k] = sum over the block's entries of U[j][k] * r[j], k < 4
__global__ void __launch_bounds__(256) ut_dot_kernel(const double* __restrict__ U,
                                                     const double* __restrict__ r, ll n,
                                                     double* __restrict__ partial, const int* stop) {
  if (stopped(stop)) return;
  __shared__ double sh[32];
  double acc[RK] = {0, 0, 0, 0};
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x) {
    const double rv = r[e];
#pragma unroll
    for (int k = 0; k < RK; ++k) acc[k] = fma(U[e * RK + k], rv, acc[k]);
  }
#pragma unroll
  for (int k = 0; k < RK; ++k) {
    const double s = block_sum(acc[k], sh);
    if (threadIdx.x == 0) partial[(ll)blockIdx.x * RK + k] = s;
  }
}

// w[k] = sum_b partial[b][k] (one block per k, fixed order)
__global__ void ut_reduce_kernel(const double* __restrict__ partial, int nblk,
                                 double* __restrict__ w, const int* stop) {
  if (stopped(stop)) return;
  __shared__ double sh[32];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(ll)b * RK + k];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) w[k] = s;
}

// z = p * r + U w
__global__ void precond_apply_kernel(const double* __restrict__ p, const double* __restrict__ U,
                                     const double* __restrict__ w, const double* __restrict__ r,
                                     double* __restrict__ z, ll n, const int* stop) {
  if (stopped(stop)) return;
  const double w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3];
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x) {
    const double* u = U + e * RK;
    z[e] = p[e] * r[e] + u[0] * w0 + u[1] * w1 + u[2] * w2 + u[3] * w3;
  }
}

// e = x* - (p * b + U w)
__global__ void residual_error_kernel(const double* __restrict__ p, const double* __restrict__ U,
                                      const double* __restrict__ w, const double* __restrict__ b,
                                      const double* __restrict__ xs, double* __restrict__ e_out, ll n) {
  const double w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3];
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x) {
    const double* u = U + e * RK;
    e_out[e] = xs[e] - (p[e] * b[e] + u[0] * w0 + u[1] * w1 + u[2] * w2 + u[3] * w3);
  }
}

// partial dot products: (x* . b, e . Ae)
__global__ void __launch_bounds__(256) dot2_kernel(const double* a0, const double* b0, const double* a1,
                                                   const double* b1, ll n, double* partial) {
  __shared__ double sh[32];
  double s0 = 0, s1 = 0;
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x) {
    s0 = fma(a0[e], b0[e], s0);
    s1 = fma(a1[e], b1[e], s1);
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 2] = s0;
    partial[blockIdx.x * 2 + 1] = s1;
  }
}

__global__ void reduce2_kernel(const double* partial, int nblk, double* out /* D, eAe */,
                               double* loss_accum) {
  __shared__ double sh[32];
  double s0 = 0, s1 = 0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    s0 += partial[b * 2];
    s1 += partial[b * 2 + 1];
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    out[0] = s0;
    out[1] = s1;
    if (loss_accum) *loss_accum += s1 / s0;
  }
}

// g = -2 Ae / D (in place over Ae)
__global__ void scale_g_kernel(double* __restrict__ Ae, const double* __restrict__ DeAe, ll n) {
  const double f = -2.0 / DeAe[0];
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x)
    Ae[e] *= f;
}

// per entry: dO from g, then backprop through the layers; stores
// H1, H2 (activations) and DA1, DA2, DO (pre-activation gradients)
__global__ void __launch_bounds__(MT) backward_entry_kernel(
    const float* __restrict__ params, const float* __restrict__ X, const float* __restrict__ O,
    const double* __restrict__ diag, const double* __restrict__ g, const double* __restrict__ b,
    const double* __restrict__ wb /* U^T b */, const double* __restrict__ wg /* U^T g */, ll n,
    float* __restrict__ H1, float* __restrict__ H2, float* __restrict__ DA1,
    float* __restrict__ DA2, float* __restrict__ DO) {
  __shared__ float sP[NP];
  load_params(params, sP);
  const double inv_sqrt_n = 1.0 / sqrt((double)n);
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x) {
    float x[F];
#pragma unroll
    for (int k = 0; k < F; ++k) x[k] = X[e * F + k];
    float h1[H], h2[H], o[NO];
    forward_entry(sP, x, h1, h2, o);
    const double ge = g[e], be = b[e];
    float dout[NO];
    dout[0] = (float)(ge * be * (double)sigmoid_f(O[e * NO]) / diag[e]);
#pragma unroll
    for (int k = 0; k < RK; ++k) dout[1 + k] = (float)((ge * wb[k] + be * wg[k]) * inv_sqrt_n);
#pragma unroll
    for (int j = 0; j < NO; ++j) DO[e * NO + j] = dout[j];
    // da2_i = (sum_j W3[j][i] dout_j) (1 - h2_i^2)
    float da2[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < NO; ++j) acc = fmaf(sP[OW3 + j * H + i], dout[j], acc);
      da2[i] = acc * (1.f - h2[i] * h2[i]);
      H1[e * H + i] = h1[i];
      H2[e * H + i] = h2[i];
      DA2[e * H + i] = da2[i];
    }
    // da1_k = (sum_i W2[i][k] da2_i) (1 - h1_k^2)
#pragma unroll 4
    for (int k = 0; k < H; ++k) {
      float acc = 0.f;
#pragma unroll
      for (int i = 0; i < H; ++i) acc = fmaf(sP[OW2 + i * H + k], da2[i], acc);
      DA1[e * H + k] = acc * (1.f - h1[k] * h1[k]);
    }
  }
}

// weight gradients, one thread per parameter, summing over entries in order:
//   dW1[i][k] = sum_e DA1[e][i] X[e][k],  db1[i] = sum_e DA1[e][i]
//   dW2[i][k] = sum_e DA2[e][i] H1[e][k], db2[i] = sum_e DA2[e][i]
//   dW3[j][i] = sum_e DO[e][j] H2[e][i],  db3[j] = sum_e DO[e][j]
// grad_out += (accumulates over systems)
__global__ void weight_grad_kernel(const float* __restrict__ X, const float* __restrict__ H1,
                                   const float* __restrict__ H2, const float* __restrict__ DA1,
                                   const float* __restrict__ DA2, const float* __restrict__ DO, ll n,
                                   float* __restrict__ grad) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NP) return;
  const float *G, *A;
  int gi, ai, gs, as;
  if (q < OB1) { G = DA1; gs = H; gi = (q - OW1) / F; A = X; as = F; ai = (q - OW1) % F; }
  else if (q < OW2) { G = DA1; gs = H; gi = q - OB1; A = nullptr; as = 0; ai = 0; }
  else if (q < OB2) { G = DA2; gs = H; gi = (q - OW2) / H; A = H1; as = H; ai = (q - OW2) % H; }
  else if (q < OW3) { G = DA2; gs = H; gi = q - OB2; A = nullptr; as = 0; ai = 0; }
  else if (q < OB3) { G = DO; gs = NO; gi = (q - OW3) / H; A = H2; as = H; ai = (q - OW3) % H; }
  else { G = DO; gs = NO; gi = q - OB3; A = nullptr; as = 0; ai = 0; }
  double acc = 0.0;
  for (ll e = 0; e < n; ++e) {
    const double gv = (double)G[e * gs + gi];
    acc += A ? gv * (double)A[e * as + ai] : gv;
  }
  grad[q] += (float)acc;
}

__global__ void adam_kernel(float* __restrict__ params, const float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v, int t, float lr,
                            float beta1, float beta2, float eps, float gscale) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NP) return;
  const float g = grad[q] * gscale;
  const float mq = beta1 * m[q] + (1.f - beta1) * g;
  const float vq = beta2 * v[q] + (1.f - beta2) * g * g;
  m[q] = mq;
  v[q] = vq;
  const float mh = mq / (1.f - powf(beta1, (float)t));
  const float vh = vq / (1.f - powf(beta2, (float)t));
  params[q] -= lr * mh / (sqrtf(vh) + eps);
}

int ew_grid(const seemps_ctx* ctx, ll n) { return stride_grid(ctx, n, 256, 4); }

}  // namespace

struct seemps_mlp {
  float* params;  // caller-owned device buffer of NP floats
  int site;
  int n_sites;
};

// prepared preconditioner of one local system (lives in the workspace)
struct MlpState {
  double* p;
  double* U;
  double* w;
  double* partial;
  int G;
  ll n;
};

static seemps_status mlp_prepare_impl(seemps_ctx* ctx, const seemps_mlp* mlp, const seemps_pair_dims* dm,
                                      const double* L, const double* R, const double* diag,
                                      MlpState* s, float** X_out, float** O_out) {
  const ll n = (ll)dm->chi_l * dm->d * dm->d * dm->chi_r;
  s->n = n;
  s->G = ew_grid(ctx, n);
  float *X, *O = nullptr;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n * F, &X));
  if (O_out) SEEMPS_TRY(ws_alloc(ctx, (size_t)n * NO, &O));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n, &s->p));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n * RK, &s->U));
  SEEMPS_TRY(ws_alloc(ctx, RK, &s->w));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)s->G * RK, &s->partial));
  features_kernel<<<ew_grid(ctx, n), 256, 0, ctx->stream>>>(diag, L, R, dm->chi_l, dm->chi_r, dm->d,
                                                             dm->D_l, dm->D_r, mlp->site, mlp->n_sites, X);
  SEEMPS_LAUNCHED(ctx);
  forward_kernel<<<stride_grid(ctx, n, MT, 4), MT, 0, ctx->stream>>>(mlp->params, X, diag, n, s->p, s->U, O);
  SEEMPS_LAUNCHED(ctx);
  if (X_out) *X_out = X;
  if (O_out) *O_out = O;
  return SEEMPS_OK;
}

static seemps_status mlp_apply_impl(seemps_ctx* ctx, const MlpState* s, const double* r, double* z,
                                    const int* skip) {
  ut_dot_kernel<<<s->G, 256, 0, ctx->stream>>>(s->U, r, s->n, s->partial, skip);
  ut_reduce_kernel<<<RK, 256, 0, ctx->stream>>>(s->partial, s->G, s->w, skip);
  precond_apply_kernel<<<s->G, 256, 0, ctx->stream>>>(s->p, s->U, s->w, r, z, s->n, skip);
  ctx->launches += 3;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    seemps_set_error(ctx, "mlp apply: %s", cudaGetErrorString(e));
    return SEEMPS_ERR_CUDA;
  }
  return SEEMPS_OK;
}

// hooks used by the PCG solver (krylov.cu); `storage` is host memory of at
// least mlp_state_bytes() bytes that outlives the solve.
size_t mlp_state_bytes() { return sizeof(MlpState); }

seemps_status mlp_precond_prepare(seemps_ctx* ctx, const seemps_mlp* mlp, const seemps_pair_dims* dm,
                                  int site, int n_sites, const double* L, const double* R,
                                  const double* diag, void* storage) {
  seemps_mlp local = *mlp;
  if (site >= 0) {
    local.site = site;
    local.n_sites = n_sites;
  }
  return mlp_prepare_impl(ctx, &local, dm, L, R, diag, (MlpState*)storage, nullptr, nullptr);
}

seemps_status mlp_precond_apply(seemps_ctx* ctx, void* storage, const double* r, double* z,
                                const int* skip) {
  return mlp_apply_impl(ctx, (const MlpState*)storage, r, z, skip);
}

// ----------------------------------------------------------------- C ABI
extern "C" seemps_status seemps_mlp_param_count(int hidden, int* count) {
  if (!count || hidden != H) return SEEMPS_ERR_INVALID;
  *count = NP;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_mlp_create(seemps_mlp** out, int hidden, float* params) {
  if (!out || !params || hidden != H) return SEEMPS_ERR_INVALID;
  seemps_mlp* m = new seemps_mlp;
  m->params = params;
  m->site = 0;
  m->n_sites = 1;
  *out = m;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_mlp_destroy(seemps_mlp* mlp) {
  delete mlp;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_mlp_set_site(seemps_mlp* mlp, int site, int n_sites) {
  if (!mlp || n_sites < 1 || site < 0 || site >= n_sites) return SEEMPS_ERR_INVALID;
  mlp->site = site;
  mlp->n_sites = n_sites;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_mlp_forward(seemps_ctx* ctx, const seemps_mlp* mlp,
                                            const seemps_pair_dims* dm, const double* L,
                                            const double* W1, const double* W2, const double* R,
                                            double* p_out, double* U_out) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, mlp && dm && L && W1 && W2 && R && p_out && U_out, "mlp_forward: null argument");
  WsFrame frame(ctx);
  const ll n = (ll)dm->chi_l * dm->d * dm->d * dm->chi_r;
  double* diag;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n, &diag));
  SEEMPS_TRY(seemps_heff_diagonal(ctx, dm, L, W1, W2, R, diag));
  MlpState s;
  SEEMPS_TRY(mlp_prepare_impl(ctx, mlp, dm, L, R, diag, &s, nullptr, nullptr));
  SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(p_out, s.p, n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(U_out, s.U, n * RK * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_mlp_loss_grad(seemps_ctx* ctx, const seemps_mlp* mlp,
                                              const seemps_pair_dims* dm, const double* L,
                                              const double* W1, const double* W2, const double* R,
                                              const double* b, const double* xstar, float* grad_accum,
                                              double* loss_accum) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, mlp && dm && L && W1 && W2 && R && b && xstar && grad_accum,
                 "mlp_loss_grad: null argument");
  WsFrame frame(ctx);
  const ll n = (ll)dm->chi_l * dm->d * dm->d * dm->chi_r;
  double *diag, *e, *Ae, *wg, *scal, *partial2;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n, &diag));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n, &e));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n, &Ae));
  SEEMPS_TRY(ws_alloc(ctx, RK, &wg));
  SEEMPS_TRY(ws_alloc(ctx, 2, &scal));
  SEEMPS_TRY(seemps_heff_diagonal(ctx, dm, L, W1, W2, R, diag));
  MlpState s;
  float *X, *O;
  SEEMPS_TRY(mlp_prepare_impl(ctx, mlp, dm, L, R, diag, &s, &X, &O));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)s.G * 2, &partial2));
  // w = U^T b ; e = x* - P b ; Ae
  ut_dot_kernel<<<s.G, 256, 0, ctx->stream>>>(s.U, b, n, s.partial, nullptr);
  ut_reduce_kernel<<<RK, 256, 0, ctx->stream>>>(s.partial, s.G, s.w, nullptr);
  residual_error_kernel<<<s.G, 256, 0, ctx->stream>>>(s.p, s.U, s.w, b, xstar, e, n);
  ctx->launches += 3;
  HeffPlan plan;
  SEEMPS_TRY(heff_plan(ctx, dm, L, W1, W2, R, SEEMPS_FP64, &plan));
  SEEMPS_TRY(heff_run(ctx, &plan, e, Ae));
  // D = x*.b, eAe ; loss += eAe / D ; g = -2 Ae / D ; U^T g
  dot2_kernel<<<s.G, 256, 0, ctx->stream>>>(xstar, b, e, Ae, n, partial2);
  reduce2_kernel<<<1, 256, 0, ctx->stream>>>(partial2, s.G, scal, loss_accum);
  scale_g_kernel<<<s.G, 256, 0, ctx->stream>>>(Ae, scal, n);
  ut_dot_kernel<<<s.G, 256, 0, ctx->stream>>>(s.U, Ae, n, s.partial, nullptr);
  ut_reduce_kernel<<<RK, 256, 0, ctx->stream>>>(s.partial, s.G, wg, nullptr);
  ctx->launches += 5;
  float *H1, *H2, *DA1, *DA2, *DO;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n * H, &H1));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n * H, &H2));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n * H, &DA1));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n * H, &DA2));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n * NO, &DO));
  backward_entry_kernel<<<stride_grid(ctx, n, MT, 4), MT, 0, ctx->stream>>>(
      mlp->params, X, O, diag, Ae, b, s.w, wg, n, H1, H2, DA1, DA2, DO);
  SEEMPS_LAUNCHED(ctx);
  weight_grad_kernel<<<ceil_div(NP, 128), 128, 0, ctx->stream>>>(X, H1, H2, DA1, DA2, DO, n, grad_accum);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_mlp_adam(seemps_ctx* ctx, seemps_mlp* mlp, const float* grad, float* m,
                                         float* v, int t, float lr, float beta1, float beta2, float eps,
                                         float grad_scale) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, mlp && grad && m && v && t >= 1, "mlp_adam: bad argument");
  adam_kernel<<<ceil_div(NP, 256), 256, 0, ctx->stream>>>(mlp->params, grad, m, v, t, lr, beta1, beta2,
                                                            eps, grad_scale);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

// Adam training on a set of local systems: per step the mean loss and
// gradient over a mini-batch (systems taken cyclically), then one Adam
// update; the Adam step counter continues from *t_inout.
extern "C" seemps_status seemps_mlp_train(seemps_ctx* ctx, seemps_mlp* mlp, const seemps_mlp_dataset* ds,
                                          const seemps_mlp_train_params* tp, float* grad, float* m, float* v,
                                          int* t_inout, double* loss_history) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, mlp && ds && tp && grad && m && v && t_inout, "mlp_train: null argument");
  SEEMPS_REQUIRE(ctx, ds->n_systems >= 1 && ds->dims && ds->L && ds->W1 && ds->W2 && ds->R && ds->b &&
                          ds->xstar && ds->site && ds->n_sites,
                 "mlp_train: incomplete dataset");
  SEEMPS_REQUIRE(ctx, tp->steps >= 0 && tp->lr > 0.f && *t_inout >= 0, "mlp_train: bad parameters");
  const int n = ds->n_systems;
  const int bsz = (tp->batch <= 0 || tp->batch > n) ? n : tp->batch;
  WsFrame frame(ctx);
  double* loss;
  SEEMPS_TRY(ws_alloc(ctx, 1, &loss));
  int t = *t_inout;
  for (int step = 0; step < tp->steps; ++step) {
    SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(grad, 0, sizeof(float) * NP, ctx->stream));
    SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(loss, 0, sizeof(double), ctx->stream));
    for (int k = 0; k < bsz; ++k) {
      const int q = (int)(((ll)step * bsz + k) % n);
      seemps_mlp local = *mlp;
      SEEMPS_REQUIRE(ctx, ds->n_sites[q] >= 1 && ds->site[q] >= 0 && ds->site[q] < ds->n_sites[q],
                     "mlp_train: bad site of system %d", q);
      local.site = ds->site[q];
      local.n_sites = ds->n_sites[q];
      SEEMPS_TRY(seemps_mlp_loss_grad(ctx, &local, &ds->dims[q], ds->L[q], ds->W1[q], ds->W2[q], ds->R[q],
                                      ds->b[q], ds->xstar[q], grad, loss));
    }
    ++t;
    SEEMPS_TRY(seemps_mlp_adam(ctx, mlp, grad, m, v, t, tp->lr, tp->beta1, tp->beta2, tp->eps, 1.f / (float)bsz));
    if (loss_history) {
      double h = 0.0;
      SEEMPS_TRY(copy_scalar_to_host(ctx, loss, &h, sizeof(double)));
      loss_history[step] = h / bsz;
    }
  }
  *t_inout = t;
  return SEEMPS_OK;
}
