// Double-FP64 (double-double) contractions of the quadratic form: the
// environment update and the effective operator H_n a (Sect. 2.5), for
// operators whose MPO sums channels of very different size.
//
// The QTT Laplacian of Sect. 5.1 is the example: on 2^n points its MPO adds
// the identity and the two shift channels with weights of order 1/h^2 ~ 4^n,
// and their sum acting on a smooth vector is of order 1.  In FP64 every
// environment entry and every operator product then carries an absolute
// rounding error of order eps 4^n relative to the result, which bounds the
// solution error of the DMRG solve (Sect. 3.2.3) at about eps 4^n / 40
// (3e-6 at n = 20 per dimension).  Carrying the environments and the
// operator product as unevaluated sums hi + lo of two FP64 numbers (about
// 106 significant bits) removes that floor; the MPS tensors, the two-site
// vector, the local solver's vectors and the split stay FP64.
//
// Storage: a double-FP64 tensor of n elements is one buffer of 2n doubles,
// the n high parts followed by the n low parts, so that a reader that wants
// FP64 (the Jacobi diagonal, environment norms) uses the first half as is.
//
// Arithmetic: every product a b of a = ah + al and b = bh + bl enters as
// the exact product ah bh (its rounding error recovered with one FMA) plus
// ah bl + al bh; the sum is accumulated with an error-free two-sum of the
// high parts and an FP64 sum of the low parts (Dekker 1971; Knuth, TAOCP
// vol. 2, Sect. 4.2.2), renormalised once at the end.  The relative error of
// a contraction is about K eps^2 times the sum of the magnitudes of its terms.
#include "contract.cuh"
#include "timing.cuh"

namespace {

// Error-free transformations.  The _rn intrinsics keep the compiler from
// contracting the additions and the product into FMAs, which would break the
// error terms.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double z = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, z)), __dsub_rn(b, z));
}

// (sh, sl) += (ah + al) (bh + bl), the al bl term (below 2^-104 of the
// product) dropped
__device__ __forceinline__ void dd_mac(double& sh, double& sl, double ah, double al, double bh, double bl) {
  const double p = __dmul_rn(ah, bh);
  double e = fma(ah, bh, -p);  // ah bh - p exactly
  e = fma(ah, bl, e);
  e = fma(al, bh, e);
  double s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl = __dadd_rn(sl, __dadd_rn(t, e));
}

// ------------------------------------------------------------------ GEMM
// C(m, n) = sum_k A(m, k) B(k, n) with X(i, j) at X + i sX0 + j sX1; a null
// low part reads as zero; a null Cl stores the FP64 rounding of the sum.
struct DdGemmArgs {
  int M, N, K;
  const double *Ah, *Al;
  ll sAm, sAk;
  const double *Bh, *Bl;
  ll sBk, sBn;
  double *Ch, *Cl;
  ll sCm, sCn;
  const int* skip;
};

// (16 MT) x (16 MT) output tile per 256-thread block, K staged 16 at a time
// in shared memory (both parts of both operands); each thread owns an MT x MT
// strided micro-tile (rows ty + 16 i, columns tx + 16 j).  MT = 4 (64 x 64
// tiles) when that still gives a wave of blocks, else MT = 2 (32 x 32) so
// that the small GEMMs of a chi ~ 64 solve spread over more SMs (the FP64
// units of each SM bound the double-FP64 multiply-adds).
constexpr int DD_BK = 16;

template <int MT>
__global__ void __launch_bounds__(256) ddgemm_kernel(DdGemmArgs a) {
  constexpr int T = 16 * MT;
  constexpr int LOADS = T * DD_BK / 256;  // elements of each plane per thread
  if (a.skip && *(volatile const int*)a.skip) return;
  __shared__ double Ah[DD_BK][T + 1], Al[DD_BK][T + 1];
  __shared__ double Bh[DD_BK][T + 1], Bl[DD_BK][T + 1];
  const int m0 = blockIdx.y * T, n0 = blockIdx.x * T;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const bool a_kfast = (a.sAk == 1);
  const bool b_nfast = (a.sBn == 1) || (a.sBk != 1);
  double ch[MT][MT], cl[MT][MT];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < MT; ++j) ch[i][j] = cl[i][j] = 0.0;

  for (int k0 = 0; k0 < a.K; k0 += DD_BK) {
#pragma unroll
    for (int q = 0; q < LOADS; ++q) {
      const int e = t + 256 * q;
      int mm, kk;
      if (a_kfast) { kk = e & 15; mm = e >> 4; } else { mm = e % T; kk = e / T; }
      int gm = m0 + mm, gk = k0 + kk;
      const bool ain = gm < a.M && gk < a.K;
      const ll ao = (ll)gm * a.sAm + (ll)gk * a.sAk;
      Ah[kk][mm] = ain ? a.Ah[ao] : 0.0;
      Al[kk][mm] = (ain && a.Al) ? a.Al[ao] : 0.0;
      int nn;
      if (b_nfast) { nn = e % T; kk = e / T; } else { kk = e & 15; nn = e >> 4; }
      const int gn = n0 + nn;
      gk = k0 + kk;
      const bool bin = gn < a.N && gk < a.K;
      const ll bo = (ll)gk * a.sBk + (ll)gn * a.sBn;
      Bh[kk][nn] = bin ? a.Bh[bo] : 0.0;
      Bl[kk][nn] = (bin && a.Bl) ? a.Bl[bo] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < DD_BK; ++kk) {
      double ah[MT], al[MT], bh[MT], bl[MT];
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        ah[i] = Ah[kk][ty + 16 * i];
        al[i] = Al[kk][ty + 16 * i];
      }
#pragma unroll
      for (int j = 0; j < MT; ++j) {
        bh[j] = Bh[kk][tx + 16 * j];
        bl[j] = Bl[kk][tx + 16 * j];
      }
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) dd_mac(ch[i][j], cl[i][j], ah[i], al[i], bh[j], bl[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= a.M) continue;
#pragma unroll
    for (int j = 0; j < MT; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= a.N) continue;
      double h, l;
      two_sum(ch[i][j], cl[i][j], h, l);
      const ll off = (ll)gm * a.sCm + (ll)gn * a.sCn;
      a.Ch[off] = h;
      if (a.Cl) a.Cl[off] = l;
    }
  }
}

seemps_status ddgemm(seemps_ctx* ctx, DdGemmArgs a) {
  if (a.M <= 0 || a.N <= 0) return SEEMPS_OK;
  if (a.K <= 0) {
    seemps_set_error(ctx, "ddgemm: K = %d", a.K);
    return SEEMPS_ERR_INVALID;
  }
  const bool big = (ll)ceil_div(a.N, 64) * ceil_div(a.M, 64) >= ctx->sm_count;
  const int T = big ? 64 : 32;
  dim3 grid(ceil_div(a.N, T), ceil_div(a.M, T));
  if (grid.y > 65535) {
    seemps_set_error(ctx, "ddgemm: grid too large (M = %d)", a.M);
    return SEEMPS_ERR_INVALID;
  }
  a.skip = ctx->skip;
  if (big) ddgemm_kernel<4><<<grid, 256, 0, ctx->stream>>>(a);
  else ddgemm_kernel<2><<<grid, 256, 0, ctx->stream>>>(a);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

// ------------------------------------------------------------------ MPO mixing
// One thread per (outer, inner) pair: its IN double-FP64 inputs in registers
// (NI >= IN), all OUT outputs formed from the FP64 mixing matrix (broadcast
// from shared memory).  Loads and stores are coalesced along `inner`.
constexpr int DD_MIX_NT = 128;

template <int NI>
__global__ void __launch_bounds__(DD_MIX_NT) mix_dd_kernel(MixArgs a, const double* __restrict__ in_h,
                                                           const double* __restrict__ in_l,
                                                           const double* __restrict__ Wmat,
                                                           double* __restrict__ out_h,
                                                           double* __restrict__ out_l, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  extern __shared__ __align__(16) unsigned char dd_smem[];
  double* Ws = reinterpret_cast<double*>(dd_smem);  // [IN][OUT]
  ll* ioff = reinterpret_cast<ll*>(Ws + (size_t)a.IN * a.OUT);
  ll* ooff = ioff + a.IN;
  for (int e = threadIdx.x; e < a.IN * a.OUT; e += DD_MIX_NT) Ws[e] = Wmat[e];
  for (int i = threadIdx.x; i < a.IN; i += DD_MIX_NT)
    ioff[i] = (ll)(i / a.in_n2) * a.in_s1 + (ll)(i % a.in_n2) * a.in_s2;
  for (int o = threadIdx.x; o < a.OUT; o += DD_MIX_NT)
    ooff[o] = (ll)(o / a.out_m2) * a.out_t1 + (ll)(o % a.out_m2) * a.out_t2;
  __syncthreads();
  const int inner = blockIdx.x * DD_MIX_NT + threadIdx.x;
  if (inner >= a.n_inner) return;
  const int outer = blockIdx.y;
  const ll ib = (ll)outer * a.in_so + inner;
  double xh[NI], xl[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    xh[i] = i < a.IN ? in_h[ib + ioff[i]] : 0.0;
    xl[i] = i < a.IN ? in_l[ib + ioff[i]] : 0.0;
  }
  const ll ob = (ll)outer * a.out_so + (ll)inner * a.out_ti;
  for (int o = 0; o < a.OUT; ++o) {
    double sh = 0.0, sl = 0.0;
#pragma unroll
    for (int i = 0; i < NI; ++i)
      if (i < a.IN) {
        const double w = Ws[i * a.OUT + o];
        if (w != 0.0) dd_mac(sh, sl, w, 0.0, xh[i], xl[i]);
      }
    double h, l;
    two_sum(sh, sl, h, l);
    out_h[ob + ooff[o]] = h;
    out_l[ob + ooff[o]] = l;
  }
}

// Wide MPO blocks (IN above the register budget): inputs read from global
// memory for every output.
__global__ void __launch_bounds__(DD_MIX_NT) mix_dd_wide_kernel(MixArgs a, const double* __restrict__ in_h,
                                                                const double* __restrict__ in_l,
                                                                const double* __restrict__ Wmat,
                                                                double* __restrict__ out_h,
                                                                double* __restrict__ out_l, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  const int inner = blockIdx.x * DD_MIX_NT + threadIdx.x;
  if (inner >= a.n_inner) return;
  const int outer = blockIdx.y;
  const ll ib = (ll)outer * a.in_so + inner;
  const ll ob = (ll)outer * a.out_so + (ll)inner * a.out_ti;
  for (int o = 0; o < a.OUT; ++o) {
    double sh = 0.0, sl = 0.0;
    for (int i = 0; i < a.IN; ++i) {
      const double w = Wmat[(ll)i * a.OUT + o];
      if (w == 0.0) continue;
      const ll off = ib + (ll)(i / a.in_n2) * a.in_s1 + (ll)(i % a.in_n2) * a.in_s2;
      dd_mac(sh, sl, w, 0.0, in_h[off], in_l[off]);
    }
    double h, l;
    two_sum(sh, sl, h, l);
    const ll off = ob + (ll)(o / a.out_m2) * a.out_t1 + (ll)(o % a.out_m2) * a.out_t2;
    out_h[off] = h;
    out_l[off] = l;
  }
}

seemps_status launch_mix_dd(seemps_ctx* ctx, const MixArgs& a, const double* in_h, const double* in_l,
                            const double* Wmat, double* out_h, double* out_l) {
  if (a.n_outer <= 0 || a.n_inner <= 0) return SEEMPS_OK;
  if (a.n_outer > 65535) {
    seemps_set_error(ctx, "mix: outer extent %d too large", a.n_outer);
    return SEEMPS_ERR_INVALID;
  }
  dim3 grid(ceil_div(a.n_inner, DD_MIX_NT), a.n_outer);
  const size_t smem = (size_t)a.IN * a.OUT * sizeof(double) + (size_t)(a.IN + a.OUT) * sizeof(ll);
  if (a.IN <= 32 && smem <= 48 * 1024) {
    if (a.IN <= 8)
      mix_dd_kernel<8><<<grid, DD_MIX_NT, smem, ctx->stream>>>(a, in_h, in_l, Wmat, out_h, out_l, ctx->skip);
    else if (a.IN <= 16)
      mix_dd_kernel<16><<<grid, DD_MIX_NT, smem, ctx->stream>>>(a, in_h, in_l, Wmat, out_h, out_l, ctx->skip);
    else
      mix_dd_kernel<32><<<grid, DD_MIX_NT, smem, ctx->stream>>>(a, in_h, in_l, Wmat, out_h, out_l, ctx->skip);
  } else {
    mix_dd_wide_kernel<<<grid, DD_MIX_NT, 0, ctx->stream>>>(a, in_h, in_l, Wmat, out_h, out_l, ctx->skip);
  }
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

}  // namespace

// y = H_n theta with double-FP64 environments L, R (hi parts followed by lo
// parts) and FP64 theta, y: T1 = L . theta (sum over a), mix with W1 W2 (sum
// over b, s, t), y = T2 . R (sum over f, c), rounded to FP64 once at the end.
seemps_status heff_run_dd(seemps_ctx* ctx, const HeffPlan* p, const double* theta, double* y) {
  const int chil = p->dm.chi_l, chir = p->dm.chi_r, Dl = p->dm.D_l, Dr = p->dm.D_r;
  const int kl = p->kl, kr = p->kr;
  const int d2 = p->dp;
  const ll nL = (ll)chil * Dl * kl, nR = (ll)chir * Dr * kr;
  const ll t1n = (ll)chil * Dl * d2 * kr, t2n = (ll)chil * d2 * Dr * kr;
  double *T1l = p->T1 + t1n, *T2l = p->T2 + t2n;
  DdGemmArgs g1 = {chil * Dl, d2 * kr, kl, p->L, p->L + nL, kl, 1, theta, nullptr, (ll)d2 * kr, 1,
                   p->T1, T1l, (ll)d2 * kr, 1, nullptr};
  SEEMPS_TRY(ddgemm(ctx, g1));
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
  const ll ld2 = (ll)Dr * kr;
  mx.out_so = d2 * ld2;
  mx.out_t1 = ld2;
  mx.out_t2 = kr;
  SEEMPS_TRY(launch_mix_dd(ctx, mx, p->T1, T1l, p->Wmat, p->T2, T2l));
  DdGemmArgs g3 = {chil * d2, chir, Dr * kr, p->T2, T2l, ld2, 1, p->R, p->R + nR, 1, ld2,
                   y, nullptr, chir, 1, nullptr};
  return ddgemm(ctx, g3);
}

// E_out (double-FP64) from E_in (double-FP64), the bra tensor X, the MPO
// tensor W (as the mixing matrix Wmat) and the ket tensor B (both FP64): the
// same three steps as the FP64 update, with mx the mixing layout of the side.
seemps_status env_update_dd(seemps_ctx* ctx, int side, int cix, int cib, int cox, int cob, int d, int Di,
                            int Do, const double* E_in, const double* X, const double* B, const double* Wmat,
                            MixArgs mx, double* E_out) {
  const bool right = (side == SEEMPS_RIGHT);
  const ll xrows = (ll)d * cox, xcols = (ll)Di * cib;
  const ll zcols = (ll)cib * d;
  const ll nin = (ll)cix * Di * cib, nout = (ll)cox * Do * cob;
  double *X1, *Z;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)(2 * xrows * xcols), &X1));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)(2 * cox * Do * zcols), &Z));
  double* X1l = X1 + xrows * xcols;
  double* Zl = Z + (ll)cox * Do * zcols;
  if (!right) {
    // X1[(s', c'), (b, a)] = sum_a' X[a', (s', c')] E_in[a', (b, a)]
    DdGemmArgs g1 = {d * cox, Di * cib, cix, X, nullptr, 1, (ll)d * cox, E_in, E_in + nin, xcols, 1,
                     X1, X1l, xcols, 1, nullptr};
    SEEMPS_TRY(ddgemm(ctx, g1));
  } else {
    // X1[(a', s'), (f, c)] = sum_c' X[(a', s'), c'] E_in[c', (f, c)]
    DdGemmArgs g1 = {cox * d, Di * cib, cix, X, nullptr, cix, 1, E_in, E_in + nin, xcols, 1,
                     X1, X1l, xcols, 1, nullptr};
    SEEMPS_TRY(ddgemm(ctx, g1));
  }
  mx.out_so = (ll)Do * zcols;
  mx.out_t1 = zcols;
  SEEMPS_TRY(launch_mix_dd(ctx, mx, X1, X1l, Wmat, Z, Zl));
  if (!right) {
    DdGemmArgs g2 = {cox * Do, cob, cib * d, Z, Zl, zcols, 1, B, nullptr, cob, 1, E_out, E_out + nout, cob, 1,
                     nullptr};
    return ddgemm(ctx, g2);
  }
  DdGemmArgs g2 = {cox * Do, cob, d * cib, Z, Zl, zcols, 1, B, nullptr, 1, (ll)d * cib, E_out, E_out + nout,
                   cob, 1, nullptr};
  return ddgemm(ctx, g2);
}
