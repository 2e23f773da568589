// The two-site sweep (Sect. 2.5): pairs 0..N-2 left to right, then N-2..0
// right to left.  Eigen mode is two-site DMRG (Sect. 3.1.1), solve mode is
// DMRG as a linear solver (Sect. 3.2.3), simplify mode is the variational
// compression of Sect. 2.3 (the MPS of bond dimension <= chi_max closest to
// b): with x in canonical form around the pair, |x - b|^2 is a quadratic
// form in a_n whose matrix is the identity (Sect. 2.5), so its minimiser is
// the antilinear-form vector b_n itself.  Each pair update is
//   a_n = A_n A_{n+1}  ->  local solve (Lanczos or PCG on H_n; a_n = b_n)
//   ->  truncated SVD split  ->  centre move and environment update.
// The host drives the pairs; the only host reads per pair are the new bond
// dimension (it sizes the next launches) and the local solver's counters.
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "contract.cuh"
#include "timing.cuh"

namespace {

struct SweepScratch {
  double* theta;
  double* bvec;
  double* energy;
  double* resid;
  double* disc;
  int* iters;
  int* rank;
  double* norm_partial;
};

__global__ void set_one_kernel(double* p) {
  if (threadIdx.x == 0 && blockIdx.x == 0) p[0] = 1.0;
}

// the boundary environment 1 in double-FP64 storage: hi part 1, lo part 0
__global__ void set_one_dd_kernel(double* p) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    p[0] = 1.0;
    p[1] = 0.0;
  }
}

// x *= 1/sqrt(sum x^2) over one small tensor (one block)
__global__ void normalize_small_kernel(double* x, ll n) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (ll e = threadIdx.x; e < n; e += blockDim.x) acc = fma(x[e], x[e], acc);
  acc = block_sum(acc, sh);
  const double s = acc > 0.0 ? 1.0 / sqrt(acc) : 1.0;
  for (ll e = threadIdx.x; e < n; e += blockDim.x) x[e] *= s;
}

struct HostCounters {
  int rank;
  int iters;
  double energy;
  double disc;
};

seemps_status read_counters(seemps_ctx* ctx, const SweepScratch& s, HostCounters* h) {
  SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(&h->rank, s.rank, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(&h->iters, s.iters, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(&h->energy, s.energy, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(&h->disc, s.disc, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SEEMPS_OK;
}

__global__ void scale_small_kernel(double* x, ll n, double f) {
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x) x[e] *= f;
}

// Right-canonical form with the centre on site 0 (Sect. 2.3): for
// i = N-1..1 split A_i = (U S) V^T, keep V^T on site i and absorb U S into
// site i-1.  The absorbed factor is U S / |S_r| (unit norm), so that no
// intermediate grows with the chain length (an unnormalised input can
// otherwise leave the FP32 / bf16 range of the mixed-precision path); the
// product of the |S_r| is kept in log form on the host.  Eigen mode then
// normalises the centre; the other modes multiply it by that product.
seemps_status canonicalize(seemps_ctx* ctx, seemps_chain* c, const seemps_strategy* st, bool normalize,
                           int precision, const SweepScratch& s) {
  const int N = c->n_sites, d = c->d;
  int* chi = c->chi;
  double log_scale = 0.0;
  std::vector<double> sv;
  for (int i = N - 1; i >= 1; --i) {
    WsFrame frame(ctx);
    const int m = chi[i], n = d * chi[i + 1];
    const int p = m < n ? m : n;
    double *Ul, *tmp, *S;
    SEEMPS_TRY(ws_alloc(ctx, (size_t)m * p, &Ul));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)chi[i - 1] * d * p, &tmp));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &S));
    SEEMPS_TRY(seemps_svd_truncate(ctx, m, n, c->A[i], st, SEEMPS_ABSORB_LEFT, 1, Ul, s.theta,
                                   S, s.rank, s.disc, 0, precision));
    HostCounters h;
    SEEMPS_TRY(read_counters(ctx, s, &h));
    const int r = h.rank;
    sv.resize((size_t)r);
    SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(sv.data(), S, sizeof(double) * (size_t)r, cudaMemcpyDeviceToHost,
                                           ctx->stream));
    SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double kept = 0.0;
    for (int j = r - 1; j >= 0; --j) kept += sv[(size_t)j] * sv[(size_t)j];
    if (kept > 0.0) log_scale += 0.5 * log(kept);
    SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(c->A[i], s.theta, sizeof(double) * (size_t)r * n,
                                           cudaMemcpyDeviceToDevice, ctx->stream));
    // A_{i-1} <- A_{i-1} (U S / |S_r|): [chi_{i-1} d x m] . [m x r]
    DgemmArgs g = {chi[i - 1] * d, r, m, 1, 1.0, 0.0, c->A[i - 1], m, 1, 0, Ul, r, 1, 0, tmp, r, 1, 0};
    SEEMPS_TRY(gemm_prec(ctx, g, precision));
    SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(c->A[i - 1], tmp, sizeof(double) * (size_t)chi[i - 1] * d * r,
                                           cudaMemcpyDeviceToDevice, ctx->stream));
    chi[i] = r;
  }
  const ll n0 = (ll)chi[0] * d * chi[1];
  if (normalize) {
    normalize_small_kernel<<<1, 1024, 0, ctx->stream>>>(c->A[0], n0);
    SEEMPS_LAUNCHED(ctx);
  } else if (log_scale != 0.0) {
    scale_small_kernel<<<1, 1024, 0, ctx->stream>>>(c->A[0], n0, exp(log_scale));
    SEEMPS_LAUNCHED(ctx);
  }
  return SEEMPS_OK;
}

// Which environments a mode keeps: quadratic forms of the MPO (eigen, solve
// and TDVP modes), antilinear forms with b (solve and simplify modes).
static inline bool mode_quad(int mode) { return mode != SEEMPS_MODE_SIMPLIFY; }
static inline bool mode_lin(int mode) { return mode == SEEMPS_MODE_SOLVE || mode == SEEMPS_MODE_SIMPLIFY; }
// apply mode: the quadratic-form environments join x (bra) and b (ket)
static inline bool mode_apply(int mode) { return mode == SEEMPS_MODE_APPLY; }

// Left environments L_0 .. L_first and right ones R_N .. R_{first+2}.
// Quadratic-form environment across site i: left (L_i -> L_{i+1}) or right
// (R_{i+1} -> R_i); in apply mode between x (bra) and b (ket).
static seemps_status quad_env(seemps_ctx* ctx, seemps_chain* c, int mode, int side, int i, int precision) {
  const bool ab = mode_apply(mode);
  const int* cb = ab ? c->chib : c->chi;
  const double* Bi = ab ? c->B[i] : c->A[i];
  if (side == SEEMPS_LEFT)
    return env_update_braket(ctx, SEEMPS_LEFT, c->chi[i], cb[i], c->chi[i + 1], cb[i + 1], c->d, c->D[i],
                             c->D[i + 1], c->Lenv[i], c->A[i], Bi, c->W[i], c->Lenv[i + 1], precision);
  return env_update_braket(ctx, SEEMPS_RIGHT, c->chi[i + 1], cb[i + 1], c->chi[i], cb[i], c->d, c->D[i + 1],
                           c->D[i], c->Renv[i + 1], c->A[i], Bi, c->W[i], c->Renv[i], precision);
}

seemps_status build_envs(seemps_ctx* ctx, seemps_chain* c, int precision, int mode, int first) {
  const int N = c->n_sites, d = c->d;
  const bool quad = mode_quad(mode), solve = mode_lin(mode);
  if (quad) {
    if (precision == SEEMPS_FP64X2) {
      set_one_dd_kernel<<<1, 32, 0, ctx->stream>>>(c->Lenv[0]);
      SEEMPS_LAUNCHED(ctx);
      set_one_dd_kernel<<<1, 32, 0, ctx->stream>>>(c->Renv[N]);
    } else {
      set_one_kernel<<<1, 32, 0, ctx->stream>>>(c->Lenv[0]);
      SEEMPS_LAUNCHED(ctx);
      set_one_kernel<<<1, 32, 0, ctx->stream>>>(c->Renv[N]);
    }
    SEEMPS_LAUNCHED(ctx);
  }
  if (solve) {
    set_one_kernel<<<1, 32, 0, ctx->stream>>>(c->Fenv[0]);
    SEEMPS_LAUNCHED(ctx);
    set_one_kernel<<<1, 32, 0, ctx->stream>>>(c->Genv[N]);
    SEEMPS_LAUNCHED(ctx);
  }
  for (int i = 0; i < first; ++i) {
    if (quad) SEEMPS_TRY(quad_env(ctx, c, mode, SEEMPS_LEFT, i, precision));
    if (solve)
      SEEMPS_TRY(env_update_linear_run(ctx, SEEMPS_LEFT, c->chi[i], c->chi[i + 1], c->chib[i], c->chib[i + 1],
                                        d, c->Fenv[i], c->A[i], c->B[i], c->Fenv[i + 1], precision));
  }
  for (int i = N - 1; i >= first + 2; --i) {
    if (quad) SEEMPS_TRY(quad_env(ctx, c, mode, SEEMPS_RIGHT, i, precision));
    if (solve)
      SEEMPS_TRY(env_update_linear_run(ctx, SEEMPS_RIGHT, c->chi[i + 1], c->chi[i], c->chib[i + 1], c->chib[i],
                                        d, c->Genv[i + 1], c->A[i], c->B[i], c->Genv[i], precision));
  }
  return SEEMPS_OK;
}

// TDVP's backward step on the centre site j (environments L_j and R_{j+1}
// current): A_j <- exp(+dt/2 H^(j)) A_j, normalised.
seemps_status tdvp_backward(seemps_ctx* ctx, seemps_chain* c, const seemps_sweep_params* p, int prec, int j) {
  WsFrame frame(ctx);
  const int* chi = c->chi;
  seemps_pair_dims dm1 = {chi[j], chi[j + 1], c->d, c->D[j], c->D[j + 1], c->D[j + 1]};
  HeffPlan plan1;
  SEEMPS_TRY(heff1_plan(ctx, &dm1, c->Lenv[j], c->W[j], c->Renv[j + 1], prec, &plan1));
  const ll n1 = (ll)chi[j] * c->d * chi[j + 1];
  return expm_run(ctx, &plan1, n1, c->A[j], p->krylov_dim, p->breakdown_tol, 0.5 * p->tdvp_dt, nullptr, nullptr);
}

// One pair update on (i, i+1).  to_right: the centre moves right.
seemps_status pair_update(seemps_ctx* ctx, seemps_chain* c, const seemps_sweep_params* p, int prec,
                          int i, bool to_right, const SweepScratch& s, HostCounters* h) {
  const int d = c->d;
  int* chi = c->chi;
  const bool solve = (p->mode == SEEMPS_MODE_SOLVE);
  const bool quad = mode_quad(p->mode), lin = mode_lin(p->mode);
  WsFrame frame(ctx);
  if (!quad) {
    // simplify: the optimal pair tensor is the antilinear-form vector of b
    SEEMPS_TRY(b_effective_run(ctx, chi[i], chi[i + 2], c->chib[i], c->chib[i + 1], c->chib[i + 2], d,
                                  c->Fenv[i], c->B[i], c->B[i + 1], c->Genv[i + 2], s.theta, prec));
  } else if (mode_apply(p->mode)) {
    // MPO-MPS product: the optimal pair tensor is (W b)_n, the pair's MPO
    // action on b's two-site tensor between the environments of <x, W b>
    const int* cb = c->chib;
    SEEMPS_TRY(two_site_run(ctx, cb[i], cb[i + 1], cb[i + 2], d, c->B[i], c->B[i + 1], s.bvec, prec));
    seemps_pair_dims dm = {chi[i], chi[i + 2], d, c->D[i], c->D[i + 1], c->D[i + 2]};
    WsFrame inner(ctx);
    HeffPlan plan;
    SEEMPS_TRY(heff_plan_braket(ctx, &dm, cb[i], cb[i + 2], c->Lenv[i], c->W[i], c->W[i + 1], c->Renv[i + 2],
                                prec, &plan));
    SEEMPS_TRY(heff_run(ctx, &plan, s.bvec, s.theta));
  } else {
  seemps_pair_dims dm = {chi[i], chi[i + 2], d, c->D[i], c->D[i + 1], c->D[i + 2]};
  SEEMPS_TRY(two_site_run(ctx, chi[i], chi[i + 1], chi[i + 2], d, c->A[i], c->A[i + 1], s.theta, prec));
  const ll n = (ll)chi[i] * d * d * chi[i + 2];
  {
    WsFrame inner(ctx);
    HeffPlan plan;
    SEEMPS_TRY(heff_plan(ctx, &dm, c->Lenv[i], c->W[i], c->W[i + 1], c->Renv[i + 2], prec, &plan));
    if (p->mode == SEEMPS_MODE_TDVP) {
      // forward half step of the pair: a <- exp(-dt/2 H_(i,i+1)) a, normalised
      SEEMPS_TRY(expm_run(ctx, &plan, n, s.theta, p->krylov_dim, p->breakdown_tol, -0.5 * p->tdvp_dt, s.energy,
                          s.iters));
    } else if (!solve) {
      SEEMPS_TRY(lanczos_run(ctx, &plan, n, s.theta, p->krylov_dim, p->breakdown_tol, s.energy, s.iters));
    } else {
      SEEMPS_TRY(b_effective_run(ctx, chi[i], chi[i + 2], c->chib[i], c->chib[i + 1], c->chib[i + 2], d,
                                    c->Fenv[i], c->B[i], c->B[i + 1], c->Genv[i + 2], s.bvec, prec));
      SEEMPS_TRY(pcg_run(ctx, &plan, &dm, c->Lenv[i], c->W[i], c->W[i + 1], c->Renv[i + 2], s.bvec,
                         s.theta, p->precond, p->mlp, i, c->n_sites, p->pcg_rtol, p->pcg_maxiter,
                         s.resid, s.iters));
    }
  }
  }
  SEEMPS_TRY(seemps_svd_truncate(ctx, chi[i] * d, d * chi[i + 2], s.theta, &p->strategy,
                                 to_right ? SEEMPS_ABSORB_RIGHT : SEEMPS_ABSORB_LEFT,
                                 (p->mode == SEEMPS_MODE_EIG || p->mode == SEEMPS_MODE_TDVP) ? 1 : 0,
                                 c->A[i], c->A[i + 1], nullptr, s.rank, s.disc, 0, prec));
  SEEMPS_TRY(read_counters(ctx, s, h));
  const int r = h->rank;
  chi[i + 1] = r;
  if (to_right) {
    if (quad) SEEMPS_TRY(quad_env(ctx, c, p->mode, SEEMPS_LEFT, i, prec));
    if (lin)
      SEEMPS_TRY(env_update_linear_run(ctx, SEEMPS_LEFT, chi[i], r, c->chib[i], c->chib[i + 1], d, c->Fenv[i],
                                        c->A[i], c->B[i], c->Fenv[i + 1], prec));
    if (p->mode == SEEMPS_MODE_TDVP && i < c->n_sites - 2)
      SEEMPS_TRY(tdvp_backward(ctx, c, p, prec, i + 1));
  } else {
    if (quad) SEEMPS_TRY(quad_env(ctx, c, p->mode, SEEMPS_RIGHT, i + 1, prec));
    if (lin)
      SEEMPS_TRY(env_update_linear_run(ctx, SEEMPS_RIGHT, chi[i + 2], r, c->chib[i + 2], c->chib[i + 1], d,
                                        c->Genv[i + 2], c->A[i + 1], c->B[i + 1], c->Genv[i + 1], prec));
    if (p->mode == SEEMPS_MODE_TDVP && i > 0) SEEMPS_TRY(tdvp_backward(ctx, c, p, prec, i));
  }
  return SEEMPS_OK;
}

}  // namespace

static seemps_status alloc_scratch(seemps_ctx* ctx, const seemps_chain* c, const seemps_sweep_params* p,
                                   bool solve, SweepScratch* s) {
  int chimax = 1;
  for (int i = 0; i <= c->n_sites; ++i) chimax = c->chi[i] > chimax ? c->chi[i] : chimax;
  if (p->strategy.chi_max > chimax) chimax = p->strategy.chi_max;
  const ll nloc = (ll)chimax * c->d * c->d * chimax;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)nloc, &s->theta));
  s->bvec = nullptr;
  if (solve) SEEMPS_TRY(ws_alloc(ctx, (size_t)nloc, &s->bvec));
  if (mode_apply(p->mode)) {
    // b's two-site tensor
    int cbmax = 1;
    for (int i = 0; i <= c->n_sites; ++i) cbmax = c->chib[i] > cbmax ? c->chib[i] : cbmax;
    SEEMPS_TRY(ws_alloc(ctx, (size_t)cbmax * c->d * c->d * cbmax, &s->bvec));
  }
  SEEMPS_TRY(ws_alloc(ctx, 1, &s->energy));
  SEEMPS_TRY(ws_alloc(ctx, 1, &s->resid));
  SEEMPS_TRY(ws_alloc(ctx, 1, &s->disc));
  SEEMPS_TRY(ws_alloc(ctx, 1, &s->iters));
  SEEMPS_TRY(ws_alloc(ctx, 1, &s->rank));
  SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(s->energy, 0, sizeof(double), ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(s->iters, 0, sizeof(int), ctx->stream));
  return SEEMPS_OK;
}

static seemps_status check_chain(seemps_ctx* ctx, const seemps_chain* c, int mode) {
  SEEMPS_REQUIRE(ctx, c, "sweep: null chain");
  SEEMPS_REQUIRE(ctx, mode == SEEMPS_MODE_EIG || mode == SEEMPS_MODE_SOLVE || mode == SEEMPS_MODE_SIMPLIFY ||
                          mode == SEEMPS_MODE_TDVP || mode == SEEMPS_MODE_APPLY,
                 "sweep: unknown mode %d", mode);
  SEEMPS_REQUIRE(ctx, c->n_sites >= 2 && c->d >= 1, "sweep: need at least two sites");
  SEEMPS_REQUIRE(ctx, c->A && c->chi, "sweep: incomplete chain");
  SEEMPS_REQUIRE(ctx, c->chi[0] == 1 && c->chi[c->n_sites] == 1, "sweep: open boundary bonds must be 1");
  if (mode_quad(mode)) {
    SEEMPS_REQUIRE(ctx, c->D && c->W && c->Lenv && c->Renv, "sweep: incomplete chain (MPO, environments)");
    SEEMPS_REQUIRE(ctx, c->D[0] == 1 && c->D[c->n_sites] == 1, "sweep: open boundary MPO bonds must be 1");
  }
  if (mode_apply(mode)) {
    SEEMPS_REQUIRE(ctx, c->B && c->chib, "sweep: apply mode needs b");
    SEEMPS_REQUIRE(ctx, c->chib[0] == 1 && c->chib[c->n_sites] == 1, "sweep: open boundary bonds of b must be 1");
  }
  if (mode_lin(mode)) {
    SEEMPS_REQUIRE(ctx, c->B && c->chib && c->Fenv && c->Genv, "sweep: this mode needs b");
    SEEMPS_REQUIRE(ctx, c->chib[0] == 1 && c->chib[c->n_sites] == 1, "sweep: open boundary bonds of b must be 1");
  }
  return SEEMPS_OK;
}

// Precisions of the sweep: FP64, BF16X3, and FP64X2 (double-FP64 quadratic-
// form environments and effective operator; not for TDVP, whose one-site
// operator has no double-FP64 path).
static seemps_status check_precision(seemps_ctx* ctx, int mode, int precision) {
  SEEMPS_REQUIRE(ctx, precision == SEEMPS_FP64 || precision == SEEMPS_BF16X3 || precision == SEEMPS_FP64X2,
                 "sweep: bad precision %d", precision);
  SEEMPS_REQUIRE(ctx, !(precision == SEEMPS_FP64X2 && mode == SEEMPS_MODE_TDVP),
                 "sweep: TDVP has no double-FP64 path");
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_build_environments(seemps_ctx* ctx, seemps_chain* c, int mode, int first,
                                                   int precision) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_TRY(check_chain(ctx, c, mode));
  SEEMPS_REQUIRE(ctx, first >= 0 && first <= c->n_sites - 2, "build_environments: bad first pair");
  SEEMPS_TRY(check_precision(ctx, mode, precision));
  return build_envs(ctx, c, precision, mode, first);
}

extern "C" seemps_status seemps_sweep_range(seemps_ctx* ctx, seemps_chain* c, const seemps_sweep_params* p,
                                            int first, int count, int direction, seemps_sweep_report* rep) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, p, "sweep_range: null params");
  SEEMPS_TRY(check_chain(ctx, c, p->mode));
  SEEMPS_REQUIRE(ctx, p->mode != SEEMPS_MODE_TDVP || (p->tdvp_dt > 0.0 && p->tdvp_dt < 1e300),
                 "sweep: TDVP needs a finite time step dt > 0");
  SEEMPS_REQUIRE(ctx, direction == 1 || direction == -1, "sweep_range: direction must be +1 or -1");
  const int last = first + direction * (count - 1);
  SEEMPS_REQUIRE(ctx, count >= 0 && first >= 0 && first <= c->n_sites - 2 && last >= 0 &&
                          last <= c->n_sites - 2, "sweep_range: pairs out of range");
  SEEMPS_TRY(check_precision(ctx, p->mode, p->precision));
  auto t0 = std::chrono::steady_clock::now();
  WsFrame frame(ctx);
  SweepScratch s;
  SEEMPS_TRY(alloc_scratch(ctx, c, p, p->mode == SEEMPS_MODE_SOLVE, &s));
  HostCounters h = {0, 0, 0.0, 0.0};
  double max_disc = 0.0, err = 0.0;
  long long iters = 0;
  for (int k = 0; k < count; ++k) {
    const int i = first + direction * k;
    SEEMPS_TRY(pair_update(ctx, c, p, p->precision, i, direction > 0, s, &h));
    SEEMPS_TRY(timing_flush(ctx));
    iters += h.iters;
    err += h.disc;
    max_disc = h.disc > max_disc ? h.disc : max_disc;
  }
  SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (rep) {
    rep->energy = h.energy;
    rep->max_discarded = max_disc;
    rep->error_bound = err;
    rep->local_iters = iters;
    rep->half_sweeps = 0;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_sweep(seemps_ctx* ctx, seemps_chain* c, const seemps_sweep_params* p,
                                      seemps_sweep_report* rep) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, c && p, "sweep: null argument");
  SEEMPS_TRY(check_chain(ctx, c, p->mode));
  SEEMPS_REQUIRE(ctx, p->mode != SEEMPS_MODE_TDVP || (p->tdvp_dt > 0.0 && p->tdvp_dt < 1e300),
                 "sweep: TDVP needs a finite time step dt > 0");
  const int N = c->n_sites;
  const bool solve = (p->mode == SEEMPS_MODE_SOLVE);
  SEEMPS_TRY(check_precision(ctx, p->mode, p->precision));
  SEEMPS_REQUIRE(ctx, p->strategy.chi_max >= 1, "sweep: chi_max < 1");
  for (int i = 0; i < N; ++i) SEEMPS_REQUIRE(ctx, c->chi[i + 1] <= p->strategy.chi_max || p->canonicalize,
                                             "sweep: bond %d exceeds chi_max", i + 1);
  auto t0 = std::chrono::steady_clock::now();
  WsFrame frame(ctx);
  SweepScratch s;
  SEEMPS_TRY(alloc_scratch(ctx, c, p, solve, &s));

  if (p->canonicalize)
    SEEMPS_TRY(canonicalize(ctx, c, &p->strategy, p->mode == SEEMPS_MODE_EIG || p->mode == SEEMPS_MODE_TDVP,
                            p->precision, s));
  SEEMPS_TRY(build_envs(ctx, c, p->precision, p->mode, 0));

  double max_disc = 0.0, err = 0.0;
  long long iters = 0;
  int half = 0;
  HostCounters h = {0, 0, 0.0, 0.0};
  const int total = p->n_sweeps + p->refine_sweeps;
  for (int sw = 0; sw < total; ++sw) {
    const int prec = sw < p->n_sweeps ? p->precision : SEEMPS_FP64;
    if (sw == p->n_sweeps && sw > 0 && p->precision != SEEMPS_FP64) {
      // refinement: environments rebuilt in FP64 from the current MPS
      SEEMPS_TRY(build_envs(ctx, c, SEEMPS_FP64, p->mode, 0));
    }
    for (int dir = 0; dir < 2; ++dir) {
      int maxr = 0;
      for (int k = 0; k < N - 1; ++k) {
        const int i = dir == 0 ? k : N - 2 - k;
        SEEMPS_TRY(pair_update(ctx, c, p, prec, i, dir == 0, s, &h));
        SEEMPS_TRY(timing_flush(ctx));
        iters += h.iters;
        err += h.disc;
        max_disc = h.disc > max_disc ? h.disc : max_disc;
        maxr = h.rank > maxr ? h.rank : maxr;
      }
      if (rep && rep->half_sweep_energy) rep->half_sweep_energy[half] = h.energy;
      if (rep && rep->half_sweep_max_rank) rep->half_sweep_max_rank[half] = maxr;
      ++half;
    }
  }
  SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (rep) {
    rep->energy = h.energy;
    rep->max_discarded = max_disc;
    rep->error_bound = err;
    rep->local_iters = iters;
    rep->half_sweeps = half;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return SEEMPS_OK;
}

// Many independent chains at once: a pool of host threads takes chains from
// a shared counter; each runs seemps_sweep on the chain's own context (own
// stream and workspace), so the GPU overlaps the chains' kernels and one
// chain's per-pair host reads never stall another chain.
extern "C" seemps_status seemps_sweep_batch(seemps_ctx* const* ctxs, seemps_chain* const* chains,
                                            const seemps_sweep_params* const* params, int n_chains,
                                            int max_threads, seemps_sweep_report* reports,
                                            seemps_status* statuses) {
  if (!ctxs || !chains || !params || n_chains < 0 || !statuses) return SEEMPS_ERR_INVALID;
  for (int k = 0; k < n_chains; ++k) {
    if (!ctxs[k] || !chains[k] || !params[k]) return SEEMPS_ERR_INVALID;
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return SEEMPS_ERR_INVALID;  // one context (stream, workspace) per chain
  }
  int nt = max_threads > 0 ? max_threads : 16;
  if (nt > n_chains) nt = n_chains;
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n_chains) break;
      cudaSetDevice(ctxs[k]->device);
      statuses[k] = seemps_sweep(ctxs[k], chains[k], params[k], reports ? &reports[k] : nullptr);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  if (nt > 0) worker();
  for (auto& th : pool) th.join();
  for (int k = 0; k < n_chains; ++k)
    if (statuses[k] != SEEMPS_OK) return statuses[k];
  return SEEMPS_OK;
}
