// Global conjugate gradients on MPS (Sect. 3.2.1, the CGS listing of
// Fig. cgs) for a symmetric positive definite MPO U and an MPS b, built from
// the sweep's own pieces: the joined MPS of a weighted sum (Sect. 2.4.1),
// compressed by the simplify sweep; the product U x by the variational
// MPO-MPS product sweep (Sect. 2.4.2); norms and <p, U p> by contracting the
// linear and quadratic forms' environments along the chain (Sect. 2.5).
//
// The driver runs on the host: each step issues its sweeps on the context's
// stream and reads two scalars back (|r|, <p, U p>).  The work MPS (y = U x,
// r, p), the joined tensors and the sweeps' environments live in one
// caller-allocated arena (seemps_cgs_work_bytes); nothing is allocated here.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "contract.cuh"

namespace {

constexpr int JOIN_MAX = 4;  // terms of one joined sum

__global__ void one_kernel(double* p) {
  if (threadIdx.x == 0 && blockIdx.x == 0) p[0] = 1.0;
}

struct JoinSite {
  const double* t[JOIN_MAX];
  int tl[JOIN_MAX], tr[JOIN_MAX];  // the term's bonds at this site
  int r0[JOIN_MAX], c0[JOIN_MAX];  // offsets of the term's block
  double w[JOIN_MAX];              // weight (first site only)
};

// One site of the joined MPS: a row of blocks on the first site (weighted),
// a column on the last, block diagonal between; a single site sums.
__global__ void mps_join_kernel(JoinSite js, int K, int d, int rows, int cols, int first, int last,
                                double* __restrict__ out) {
  const ll total = (ll)rows * d * cols;
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < total; e += (ll)gridDim.x * blockDim.x) {
    const int c = (int)(e % cols), s = (int)((e / cols) % d), r = (int)(e / ((ll)cols * d));
    double v = 0.0;
    if (first && last) {
      for (int k = 0; k < K; ++k) v += js.w[k] * js.t[k][s];
    } else if (first) {
      for (int k = 0; k < K; ++k)
        if (c >= js.c0[k] && c < js.c0[k] + js.tr[k]) v = js.w[k] * js.t[k][(ll)s * js.tr[k] + (c - js.c0[k])];
    } else if (last) {
      for (int k = 0; k < K; ++k)
        if (r >= js.r0[k] && r < js.r0[k] + js.tl[k]) v = js.t[k][(ll)(r - js.r0[k]) * d + s];
    } else {
      for (int k = 0; k < K; ++k)
        if (r >= js.r0[k] && r < js.r0[k] + js.tl[k] && c >= js.c0[k] && c < js.c0[k] + js.tr[k])
          v = js.t[k][((ll)(r - js.r0[k]) * d + s) * js.tr[k] + (c - js.c0[k])];
    }
    out[e] = v;
  }
}

// An MPS held in per-site device buffers with host-side bond dimensions.
struct Mps {
  std::vector<double*> t;
  std::vector<int> chi;
};

seemps_status mps_join(seemps_ctx* ctx, int N, int d, int K, const double* w, const Mps* const* terms, Mps* out) {
  out->chi.assign(N + 1, 0);
  out->chi[0] = out->chi[N] = 1;
  for (int n = 1; n < N; ++n) {
    int s = 0;
    for (int k = 0; k < K; ++k) s += terms[k]->chi[n];
    out->chi[n] = s;
  }
  for (int n = 0; n < N; ++n) {
    JoinSite js = {};
    int r0 = 0, c0 = 0;
    for (int k = 0; k < K; ++k) {
      js.t[k] = terms[k]->t[n];
      js.tl[k] = terms[k]->chi[n];
      js.tr[k] = terms[k]->chi[n + 1];
      js.r0[k] = r0;
      js.c0[k] = c0;
      js.w[k] = w[k];
      r0 += js.tl[k];
      c0 += js.tr[k];
    }
    const int rows = out->chi[n], cols = out->chi[n + 1];
    const ll total = (ll)rows * d * cols;
    mps_join_kernel<<<stride_grid(ctx, total, 256, 4), 256, 0, ctx->stream>>>(js, K, d, rows, cols, n == 0,
                                                                                n == N - 1, out->t[n]);
    SEEMPS_LAUNCHED(ctx);
  }
  return SEEMPS_OK;
}

seemps_status mps_copy(seemps_ctx* ctx, int N, int d, const Mps& src, Mps* dst) {
  dst->chi = src.chi;
  for (int n = 0; n < N; ++n)
    SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(dst->t[n], src.t[n], sizeof(double) * src.chi[n] * d * src.chi[n + 1],
                                           cudaMemcpyDeviceToDevice, ctx->stream));
  return SEEMPS_OK;
}

// <A, B> by the antilinear form's left environments, FP64, read to the host.
seemps_status mps_overlap(seemps_ctx* ctx, int N, int d, const Mps& A, const Mps& B, double* out) {
  WsFrame frame(ctx);
  int ca = 1, cb = 1;
  for (int n = 0; n <= N; ++n) {
    ca = std::max(ca, A.chi[n]);
    cb = std::max(cb, B.chi[n]);
  }
  double *F0, *F1;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)ca * cb, &F0));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)ca * cb, &F1));
  one_kernel<<<1, 32, 0, ctx->stream>>>(F0);
  SEEMPS_LAUNCHED(ctx);
  for (int n = 0; n < N; ++n) {
    SEEMPS_TRY(env_update_linear_run(ctx, SEEMPS_LEFT, A.chi[n], A.chi[n + 1], B.chi[n], B.chi[n + 1], d, F0,
                                     A.t[n], B.t[n], F1, SEEMPS_FP64));
    std::swap(F0, F1);
  }
  SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(out, F0, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SEEMPS_OK;
}

// <A, U A> by the quadratic form's left environments, FP64, read to the host.
seemps_status mps_expectation(seemps_ctx* ctx, int N, int d, const int* D, const double* const* W, const Mps& A,
                              double* out) {
  WsFrame frame(ctx);
  int ca = 1, dm = 1;
  for (int n = 0; n <= N; ++n) {
    ca = std::max(ca, A.chi[n]);
    dm = std::max(dm, D[n]);
  }
  double *L0, *L1;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)ca * dm * ca, &L0));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)ca * dm * ca, &L1));
  one_kernel<<<1, 32, 0, ctx->stream>>>(L0);
  SEEMPS_LAUNCHED(ctx);
  for (int n = 0; n < N; ++n) {
    SEEMPS_TRY(env_update_braket(ctx, SEEMPS_LEFT, A.chi[n], A.chi[n], A.chi[n + 1], A.chi[n + 1], d, D[n],
                                 D[n + 1], L0, A.t[n], A.t[n], W[n], L1, SEEMPS_FP64));
    std::swap(L0, L1);
  }
  SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(out, L0, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SEEMPS_OK;
}

// Sizes of the arena for bond limit chi and b's bond chib.
struct CgsSizes {
  size_t cap, capT, env;  // doubles per MPS site buffer, per joined site, per environment
  int chiT;
};

CgsSizes cgs_sizes(int d, int D_max, int chi, int chib) {
  CgsSizes z;
  z.chiT = chi + std::max(chi, chib);  // the joined sums have two terms
  z.cap = (size_t)chi * d * chi;
  z.capT = (size_t)z.chiT * d * z.chiT;
  z.env = std::max((size_t)chi * z.chiT, (size_t)chi * D_max * chi);
  return z;
}

size_t cgs_bytes(int N, int d, int D_max, int chi, int chib) {
  const CgsSizes z = cgs_sizes(d, D_max, chi, chib);
  auto up = [](size_t n) { return (n * sizeof(double) + 255) & ~(size_t)255; };
  return (size_t)N * (3 * up(z.cap) + up(z.capT)) + (size_t)2 * (N + 1) * up(z.env) + 256;
}

}  // namespace

extern "C" seemps_status seemps_cgs_work_bytes(int n_sites, int d, int D_max, int chi_max, int chib_max,
                                               size_t* bytes_out) {
  if (!bytes_out || n_sites < 2 || d < 1 || D_max < 1 || chi_max < 1 || chib_max < 1) return SEEMPS_ERR_INVALID;
  *bytes_out = cgs_bytes(n_sites, d, D_max, chi_max, chib_max);
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_cgs_solve(seemps_ctx* ctx, const seemps_cgs_problem* pr,
                                          const seemps_cgs_params* prm, seemps_cgs_report* rep) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, pr && prm, "cgs: null argument");
  const int N = pr->n_sites, d = pr->d, chi = prm->strategy.chi_max;
  SEEMPS_REQUIRE(ctx, N >= 2 && d >= 1 && chi >= 1, "cgs: need n_sites >= 2, d >= 1, chi_max >= 1");
  SEEMPS_REQUIRE(ctx, pr->D && pr->W && pr->chib && pr->B && pr->chix && pr->X && pr->work,
                 "cgs: incomplete problem");
  SEEMPS_REQUIRE(ctx, prm->maxiter >= 0 && prm->n_sweeps >= 1 && prm->rtol >= 0.0, "cgs: bad parameters");
  SEEMPS_REQUIRE(ctx, prm->precision == SEEMPS_FP64 || prm->precision == SEEMPS_BF16X3, "cgs: bad precision");
  int Dmax = 1, chib = 1;
  for (int n = 0; n <= N; ++n) {
    Dmax = std::max(Dmax, pr->D[n]);
    chib = std::max(chib, pr->chib[n]);
    SEEMPS_REQUIRE(ctx, pr->chix[n] >= 1 && pr->chix[n] <= chi, "cgs: bond %d of the guess outside [1, chi_max]", n);
  }
  SEEMPS_REQUIRE(ctx, pr->work_bytes >= cgs_bytes(N, d, Dmax, chi, chib), "cgs: work arena too small");
  const auto t0 = std::chrono::steady_clock::now();

  // carve the arena
  const CgsSizes z = cgs_sizes(d, Dmax, chi, chib);
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)pr->work + 255) & ~(uintptr_t)255);
  auto take = [&](size_t n) {
    double* p = reinterpret_cast<double*>(base);
    base += (n * sizeof(double) + 255) & ~(size_t)255;
    return p;
  };
  Mps x, y, r, p, T, b;
  for (Mps* m : {&y, &r, &p}) {
    m->t.resize(N);
    for (int n = 0; n < N; ++n) m->t[n] = take(z.cap);
  }
  T.t.resize(N);
  for (int n = 0; n < N; ++n) T.t[n] = take(z.capT);
  std::vector<double*> env(2 * (N + 1));
  for (auto& e : env) e = take(z.env);
  x.t.assign(pr->X, pr->X + N);
  x.chi.assign(pr->chix, pr->chix + N + 1);
  b.t.assign(const_cast<double**>(pr->B), const_cast<double**>(pr->B) + N);
  b.chi.assign(pr->chib, pr->chib + N + 1);

  seemps_sweep_params sp = {};
  sp.n_sweeps = prm->n_sweeps;
  sp.refine_sweeps = 0;
  sp.precision = prm->precision;
  sp.krylov_dim = 2;
  sp.breakdown_tol = 1e-14;
  sp.strategy = prm->strategy;
  sp.canonicalize = 1;

  // dst <- simplify(T) from dst's current content
  auto simplify_into = [&](Mps* dst) -> seemps_status {
    seemps_chain c = {};
    c.n_sites = N;
    c.d = d;
    c.A = dst->t.data();
    c.chi = dst->chi.data();
    c.B = T.t.data();
    c.chib = T.chi.data();
    c.Fenv = env.data();
    c.Genv = env.data() + (N + 1);
    sp.mode = SEEMPS_MODE_SIMPLIFY;
    return seemps_sweep(ctx, &c, &sp, nullptr);
  };
  // y <- U x from y's current content
  auto apply_into = [&]() -> seemps_status {
    seemps_chain c = {};
    c.n_sites = N;
    c.d = d;
    c.D = pr->D;
    c.W = pr->W;
    c.A = y.t.data();
    c.chi = y.chi.data();
    c.Lenv = env.data();
    c.Renv = env.data() + (N + 1);
    c.B = x.t.data();
    c.chib = x.chi.data();
    sp.mode = SEEMPS_MODE_APPLY;
    return seemps_sweep(ctx, &c, &sp, nullptr);
  };
  auto join2 = [&](double w0, const Mps& a, double w1, const Mps& c2) -> seemps_status {
    const double w[2] = {w0, w1};
    const Mps* terms[2] = {&a, &c2};
    return mps_join(ctx, N, d, 2, w, terms, &T);
  };

  double nb2 = 0.0;
  SEEMPS_TRY(mps_overlap(ctx, N, d, b, b, &nb2));
  const double nb = sqrt(nb2 > 0.0 ? nb2 : 0.0);
  // x = simplify(guess)
  {
    const double w1[1] = {1.0};
    const Mps* t1[1] = {&x};
    SEEMPS_TRY(mps_join(ctx, N, d, 1, w1, t1, &T));
    SEEMPS_TRY(simplify_into(&x));
  }
  // r = b - U x, p = r
  SEEMPS_TRY(mps_copy(ctx, N, d, x, &y));
  SEEMPS_TRY(apply_into());
  SEEMPS_TRY(mps_copy(ctx, N, d, y, &r));
  SEEMPS_TRY(join2(1.0, b, -1.0, y));
  SEEMPS_TRY(simplify_into(&r));
  double rr = 0.0;
  SEEMPS_TRY(mps_overlap(ctx, N, d, r, r, &rr));
  double res = sqrt(rr > 0.0 ? rr : 0.0);
  SEEMPS_TRY(mps_copy(ctx, N, d, r, &p));
  if (rep && rep->residual_history) rep->residual_history[0] = res;
  int steps = 0;
  // |r| = 0 (b = 0 with x = 0, or an exact solution) is convergence whatever rtol says
  while (steps < prm->maxiter && !(res < prm->rtol * nb) && res > 0.0) {
    double pUp = 0.0;
    SEEMPS_TRY(mps_expectation(ctx, N, d, pr->D, pr->W, p, &pUp));
    SEEMPS_REQUIRE(ctx, pUp > 0.0 && isfinite(pUp), "cgs: <p, U p> = %g: U is not positive definite", pUp);
    const double alpha = res * res / pUp;
    SEEMPS_TRY(join2(1.0, x, alpha, p));
    SEEMPS_TRY(simplify_into(&x));
    SEEMPS_TRY(apply_into());
    SEEMPS_TRY(join2(1.0, b, -1.0, y));
    SEEMPS_TRY(simplify_into(&r));
    SEEMPS_TRY(mps_overlap(ctx, N, d, r, r, &rr));
    const double res_new = sqrt(rr > 0.0 ? rr : 0.0);
    const double beta = (res_new / res) * (res_new / res);
    SEEMPS_TRY(join2(1.0, r, beta, p));
    SEEMPS_TRY(simplify_into(&p));
    res = res_new;
    ++steps;
    if (rep && rep->residual_history) rep->residual_history[steps] = res;
  }
  for (int n = 0; n <= N; ++n) pr->chix[n] = x.chi[n];
  SEEMPS_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (rep) {
    rep->iterations = steps;
    rep->residual = res;
    rep->norm_b = nb;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return SEEMPS_OK;
}
