// Internal interface of the contraction layer shared by the local solvers
// and the sweep driver.
#pragma once

#include "common.cuh"

struct SplitBuf {
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
  __nv_bfloat16* lo2 = nullptr;  // third plane of the six-product GEMM
};

// Layout of one MPO mixing step: for each (outer, inner) index pair, IN
// input values map to OUT output values through a dense IN x OUT matrix.
// in_off  = outer * in_so  + (i / in_n2) * in_s1 + (i % in_n2) * in_s2 + inner
// out_off = outer * out_so + (o / out_m2) * out_t1 + (o % out_m2) * out_t2 + inner * out_ti
struct MixArgs {
  int n_outer, n_inner, IN, OUT;
  ll in_so, in_s1, in_s2;
  int in_n2;
  ll out_so, out_t1, out_t2;
  int out_m2;
  ll out_ti;
};

// Prepared operands of the effective operator of one pair: the MPO mixing
// matrix and, for bf16x3, the split copies of L and R (made once per local
// solve and reused by every apply).
struct HeffPlan {
  seemps_pair_dims dm;  // chi_l, chi_r: bonds of the output (bra) vector
  int kl, kr;    // bonds of the input (ket) vector; equal to chi_l, chi_r unless the
                 // environments join two different MPS (the MPO-MPS product)
  int dp;        // physical dimension of the vector: d^2 (two-site) or d (one-site)
  int precision;
  const double* L;
  const double* R;
  double* Wmat;  // (D_l d^2) x (d^2 D_r)
  double* T1;    // fp64 scratch
  double* T2;
  SplitBuf Ls, Rs, thT, T2s;  // bf16x3 operands and scratch
  float* T1f;
  int Kp1, Kp3;
  int fuse;  // bf16x3: the MPO mixing runs in the first GEMM's epilogue
};

seemps_status heff_plan(seemps_ctx* ctx, const seemps_pair_dims* dm, const double* L,
                        const double* W1, const double* W2, const double* R, int precision,
                        HeffPlan* p);
// The same operator between different bra and ket bonds: L (chi_l, D_l, kl),
// R (chi_r, D_r, kr); it maps (kl, d, d, kr) vectors to (chi_l, d, d, chi_r).
seemps_status heff_plan_braket(seemps_ctx* ctx, const seemps_pair_dims* dm, int kl, int kr, const double* L,
                               const double* W1, const double* W2, const double* R, int precision,
                               HeffPlan* p);
// Environment of <x, W b> (x the bra, b the ket; equal for the quadratic form):
// left: E_in (cix, D_in, cib) -> E_out (cox, D_out, cob), X (cix, d, cox), B (cib, d, cob);
// right: E_in (cix, D_in, cib) -> E_out (cox, D_out, cob), X (cox, d, cix), B (cob, d, cib).
seemps_status env_update_braket(seemps_ctx* ctx, int side, int cix, int cib, int cox, int cob, int d, int D_in,
                                int D_out, const double* E_in, const double* X, const double* B,
                                const double* W, double* E_out, int precision);
seemps_status heff_run(seemps_ctx* ctx, const HeffPlan* p, const double* theta, double* y);
// Double-FP64 pieces (dd.cu): the apply of a plan whose L and R are
// double-FP64 (precision SEEMPS_FP64X2), and the environment update with
// double-FP64 E_in / E_out given the side's mixing matrix and layout.
seemps_status heff_run_dd(seemps_ctx* ctx, const HeffPlan* p, const double* theta, double* y);
seemps_status env_update_dd(seemps_ctx* ctx, int side, int cix, int cib, int cox, int cob, int d, int Di,
                            int Do, const double* E_in, const double* X, const double* B, const double* Wmat,
                            MixArgs mx, double* E_out);
// The same apply for FP32 vectors (bf16x3 plans only): the Krylov basis of
// the mixed sweep.
seemps_status heff_run(seemps_ctx* ctx, const HeffPlan* p, const float* theta, float* y);
// One-site effective operator on a tensor (chi_l, d, chi_r) with the MPO
// tensor W (D_l, d, d, D_r); dm->D_m is ignored.  heff_run then applies it.
seemps_status heff1_plan(seemps_ctx* ctx, const seemps_pair_dims* dm, const double* L, const double* W,
                         const double* R, int precision, HeffPlan* p);
// exp(tau H) theta / |exp(tau H) theta| in the Krylov space of theta (in place);
// *alpha0 (device, may be null) receives <theta, H theta> / <theta, theta>
seemps_status expm_run(seemps_ctx* ctx, const HeffPlan* plan, ll n, double* theta, int k, double tol,
                       double tau, double* alpha0, int* iters_out);
// C = A B (alpha 1, beta 0) in the given precision (FP64 CUDA cores, or BF16X3
// tensor cores for row- or column-major operands)
seemps_status gemm_prec(seemps_ctx* ctx, const DgemmArgs& g, int precision);
// seemps_b_effective / seemps_env_update_linear in the given precision
seemps_status b_effective_run(seemps_ctx* ctx, int chi_l, int chi_r, int chib_l, int chib_m, int chib_r, int d,
                              const double* F, const double* B1, const double* B2, const double* G, double* b,
                              int precision);
seemps_status env_update_linear_run(seemps_ctx* ctx, int side, int chi_in, int chi_out, int chib_in, int chib_out,
                                    int d, const double* F_in, const double* A, const double* B, double* F_out,
                                    int precision);
// theta = A1 A2 in the given precision (FP64, or BF16X3 on the tensor cores)
seemps_status two_site_run(seemps_ctx* ctx, int chi_l, int chi_m, int chi_r, int d, const double* A1,
                           const double* A2, double* theta, int precision);
seemps_status lanczos_run(seemps_ctx* ctx, const HeffPlan* plan, ll n, double* theta, int k,
                          double tol, double* energy_out, int* iters_out);
seemps_status pcg_run(seemps_ctx* ctx, const HeffPlan* plan, const seemps_pair_dims* dm,
                      const double* L, const double* W1, const double* W2, const double* R,
                      const double* b, double* x, int precond, const seemps_mlp* mlp, int site,
                      int n_sites, double rtol, int maxiter, double* resid_out, int* iters_out);
