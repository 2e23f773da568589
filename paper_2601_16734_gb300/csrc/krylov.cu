// Local solvers of the sweep: Lanczos for the lowest eigenpair of H_n
// (Sect. 3.1.1), its Krylov exponential (Sect. 7.3, TDVP), and preconditioned
// conjugate gradients for H_n x = b (Sect. 3.2.3).  The FP64 sweep keeps
// every vector in FP64; the bf16x3 sweep stores the Krylov basis in FP32
// (its operator products carry ~2^-16 relative error) and runs the
// re-orthogonalisation in double-FP32 arithmetic (about 48 significant
// bits, error-free float products and sums): the second pass's projections,
// the work vector and the final combination (the first pass's projections
// are plain FP32 with FP64 block sums: the second pass removes what they
// leave); the scalars, the tridiagonal and the result vector are FP64.
//
// The vector kernels are bandwidth-bound: they stream the Krylov basis with
// coalesced double loads and reduce in two deterministic stages (per-block
// partials, then one block summing them in a fixed order).  Iteration
// control lives on the device (a state struct in the workspace), so no step
// needs a host round trip; a "stop" word doubles as the context's skip flag
// that turns the remaining matvec launches into no-ops.
#include <math.h>

#include <type_traits>

#include "contract.cuh"
#include "timing.cuh"

namespace {

constexpr int KMAX = 64;     // largest Krylov dimension
constexpr int VT = 256;      // threads of the vector kernels

struct LzState {
  double alpha[KMAX];
  double beta[KMAX];
  double c1[KMAX];   // first projection coefficients
  double c2[KMAX];   // second projection coefficients (alpha_j = c1[j] + c2[j])
  double y[KMAX];    // Ritz coefficients
  double norm2;
  double scale;
  double energy;
  int m;             // number of Lanczos vectors built
  int stop;          // breakdown / done flag (also the skip flag)
  int k;             // requested steps
  double tol;
};

__device__ __forceinline__ bool stopped(const int* f) { return f && *(volatile const int*)f; }

// 16-byte vector access to the Krylov basis: 4 floats or 2 doubles per load,
// so that each thread keeps several hundred bytes in flight (the vector
// kernels are bound by HBM latency x bytes in flight, not by arithmetic).
// The basis rows start on 16-byte boundaries (row stride a multiple of 32
// elements, 256-byte aligned workspace); `vec` = 0 falls back to scalar
// access for operands without that alignment (a caller's theta).
template <typename T>
using vec16_t = typename std::conditional<std::is_same<T, float>::value, float4, double2>::type;

__device__ __forceinline__ float dot_acc(const float4& a, const float4& b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}
__device__ __forceinline__ double dot_acc(const double2& a, const double2& b, double acc) {
  acc = fma(a.x, b.x, acc);
  return fma(a.y, b.y, acc);
}
__device__ __forceinline__ double sq_acc_f64(const float4& a, double acc) {
  acc = fma((double)a.x, (double)a.x, acc);
  acc = fma((double)a.y, (double)a.y, acc);
  acc = fma((double)a.z, (double)a.z, acc);
  return fma((double)a.w, (double)a.w, acc);
}
__device__ __forceinline__ double sq_acc_f64(const double2& a, double acc) { return dot_acc(a, a, acc); }
__device__ __forceinline__ void axpy_acc(float4& y, float c, const float4& v) {
  y.x = fmaf(c, v.x, y.x);
  y.y = fmaf(c, v.y, y.y);
  y.z = fmaf(c, v.z, y.z);
  y.w = fmaf(c, v.w, y.w);
}
__device__ __forceinline__ void axpy_acc(double2& y, double c, const double2& v) {
  y.x = fma(c, v.x, y.x);
  y.y = fma(c, v.y, y.y);
}

// partial[blk * ldp + i] = sum over this block's elements of V[i, n] x[n], i < nv.
// Up to DV basis vectors per pass with their accumulators in registers (x is
// read once per pass; the vectors are split evenly over the passes so that
// no pass runs with few loads in flight), then one warp-shuffle +
// shared-memory reduction per pass in a fixed order.  Products and
// per-thread sums in T, block sums in FP64.  The tail of n beyond the last
// full 16-byte vector goes to block 0.
constexpr int DV = 16;
template <typename T>
__global__ void __launch_bounds__(VT) dots_kernel(const T* __restrict__ V, ll ldv, int nv,
                                                  const T* __restrict__ x, ll n,
                                                  double* __restrict__ partial, int ldp,
                                                  const int* stop, int vec) {
  using V16 = vec16_t<T>;
  constexpr int E = 16 / sizeof(T);
  if (stopped(stop)) return;
  __shared__ double sh[VT / 32][DV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const ll nq = vec ? n / E : 0;
  const ll tail0 = nq * E;
  const int npass = (nv + DV - 1) / DV;
  const int per = (nv + npass - 1) / npass;
  for (int i0 = 0; i0 < nv; i0 += per) {
    const int cnt = nv - i0 < per ? nv - i0 : per;
    const T* Vb = V + (ll)i0 * ldv;
    T acc[DV];
#pragma unroll
    for (int c = 0; c < DV; ++c) acc[c] = T(0);
    for (ll q = blockIdx.x * (ll)VT + threadIdx.x; q < nq; q += (ll)gridDim.x * VT) {
      const V16 xv = reinterpret_cast<const V16*>(x)[q];
#pragma unroll
      for (int c = 0; c < DV; ++c)
        if (c < cnt) acc[c] = dot_acc(reinterpret_cast<const V16*>(Vb + (ll)c * ldv)[q], xv, acc[c]);
    }
    const ll e0 = vec ? tail0 + threadIdx.x : blockIdx.x * (ll)VT + threadIdx.x;
    const ll es = vec ? (ll)VT : (ll)gridDim.x * VT;
    if (!vec || blockIdx.x == 0) {
      for (ll e = e0; e < n; e += es) {
        const T xv = x[e];
#pragma unroll
        for (int c = 0; c < DV; ++c)
          if (c < cnt) acc[c] = fma(Vb[(ll)c * ldv + e], xv, acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < DV; ++c) {
      if (c < cnt) {
        const double v = warp_sum((double)acc[c]);
        if (lane == 0) sh[warp][c] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < VT / 32; ++w) t += sh[w][threadIdx.x];
      partial[(ll)blockIdx.x * ldp + i0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// x[n] -= sum_i coef[i] V[i, n]; with want_norm, also the partial squared
// norm of the new x.  V and x 16-byte aligned, ldv a multiple of 16 / sizeof(T).
template <typename T>
__global__ void __launch_bounds__(VT) update_kernel(const T* __restrict__ V, ll ldv, int nv,
                                                    const double* __restrict__ coef,
                                                    T* __restrict__ x, ll n, int want_norm,
                                                    double* __restrict__ partial, int ldp,
                                                    const int* stop) {
  using V16 = vec16_t<T>;
  constexpr int E = 16 / sizeof(T);
  if (stopped(stop)) return;
  __shared__ double sh[32];
  __shared__ T cf[KMAX];
  for (int i = threadIdx.x; i < nv; i += VT) cf[i] = -(T)coef[i];
  __syncthreads();
  const ll nq = n / E;
  T nacc = T(0);
  V16* x4 = reinterpret_cast<V16*>(x);
  for (ll q = blockIdx.x * (ll)VT + threadIdx.x; q < nq; q += (ll)gridDim.x * VT) {
    V16 v = x4[q];
#pragma unroll 8
    for (int i = 0; i < nv; ++i) axpy_acc(v, cf[i], reinterpret_cast<const V16*>(V + (ll)i * ldv)[q]);
    x4[q] = v;
    nacc = dot_acc(v, v, nacc);
  }
  if (blockIdx.x == 0) {
    for (ll e = nq * E + threadIdx.x; e < n; e += VT) {
      T v = x[e];
      for (int i = 0; i < nv; ++i) v = fma(cf[i], V[(ll)i * ldv + e], v);
      x[e] = v;
      nacc = fma(v, v, nacc);
    }
  }
  if (want_norm) {
    double s = block_sum((double)nacc, sh);
    if (threadIdx.x == 0) partial[(ll)blockIdx.x * ldp] = s;
  }
}

// out[i] = sum_b partial[b * ldp + i]: block i sums a fixed strided subset
// per thread, then a fixed-shape tree (deterministic).
__global__ void __launch_bounds__(256) reduce_kernel(const double* __restrict__ partial, int nblk,
                                                     int ldp, int nv, double* __restrict__ out,
                                                     const int* stop) {
  if (stopped(stop)) return;
  __shared__ double sh[32];
  const int i = blockIdx.x;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(ll)b * ldp + i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[i] = s;
}

// out[n] = x[n] / sqrt(*norm2), converting between the vector types
// (FP32 to FP32 scales in FP32: GB300's FP64 pipe is slow even for conversions.)
template <typename TI, typename TO>
__global__ void normalize_kernel(const TI* __restrict__ x, TO* __restrict__ out, ll n,
                                 const double* norm2, const int* stop) {
  if (stopped(stop)) return;
  const double s = 1.0 / sqrt(*norm2);
  if constexpr (std::is_same<TI, float>::value && std::is_same<TO, float>::value) {
    const float sf = (float)s;
    for (ll e = blockIdx.x * (ll)VT + threadIdx.x; e < n; e += (ll)gridDim.x * VT) out[e] = x[e] * sf;
  } else {
    for (ll e = blockIdx.x * (ll)VT + threadIdx.x; e < n; e += (ll)gridDim.x * VT)
      out[e] = (TO)((double)x[e] * s);
  }
}

// Lanczos step control after the norm of the twice-projected w is known.
__global__ void lz_control_kernel(LzState* st, int j) {
  if (threadIdx.x != 0 || st->stop) return;
  // alpha_j = the whole coefficient of v_j removed from w by the two passes
  const double a = st->c1[j] + st->c2[j];
  st->alpha[j] = a;
  const double b = sqrt(st->norm2);
  st->m = j + 1;
  const double a0 = fabs(st->alpha[0]);
  if (j == st->k - 1 || !(b > st->tol * (a0 > 1.0 ? a0 : 1.0))) {
    st->stop = 1;
  } else {
    st->beta[j] = b;
    st->scale = b * b;  // normalize_kernel divides by sqrt(scale)
  }
}

// Sturm count: number of eigenvalues of the m x m symmetric tridiagonal
// (alpha, beta) strictly below x.
__device__ int sturm_count(const double* alpha, const double* beta, int m, double x, double pivmin) {
  int cnt = 0;
  double q = alpha[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < m; ++i) {
    q = (alpha[i] - x) - beta[i - 1] * beta[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Lowest eigenpair of the tridiagonal Lanczos matrix: multisection (32
// lanes bracket the eigenvalue 33-fold per round) on the Sturm count, then
// inverse iteration with a dense partially pivoted solve in shared memory.
__global__ void tridiag_lowest_kernel(LzState* st, double* energy_out, int* iters_out) {
  __shared__ double A[KMAX][KMAX + 1];
  __shared__ double y[KMAX], rhs[KMAX];
  __shared__ double lo_s, hi_s;
  const int lane = threadIdx.x;
  const int m = st->m;
  const double* al = st->alpha;
  const double* be = st->beta;
  if (lane == 0) {
    double lo = al[0], hi = al[0], tn = 0.0;
    for (int i = 0; i < m; ++i) {
      double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i < m - 1 ? fabs(be[i]) : 0.0);
      lo = fmin(lo, al[i] - r);
      hi = fmax(hi, al[i] + r);
      tn = fmax(tn, fabs(al[i]) + r);
    }
    lo_s = lo - 1e-12 * (tn + 1.0);
    hi_s = hi + 1e-12 * (tn + 1.0);
  }
  __syncwarp();
  double lo = lo_s, hi = hi_s;
  const double tnorm = fmax(fabs(lo), fabs(hi)) + 1e-300;
  const double pivmin = 1e-300 + 1e-30 * tnorm;
  for (int round = 0; round < 40; ++round) {
    const double w = hi - lo;
    if (!(w > 2.0 * 2.2e-16 * tnorm)) break;
    const double x = lo + w * (double)(lane + 1) / 33.0;
    const int c = sturm_count(al, be, m, x, pivmin);
    const unsigned ge1 = __ballot_sync(0xffffffffu, c >= 1);  // points at or above the eigenvalue
    const int first = ge1 ? (__ffs(ge1) - 1) : 32;            // lowest such lane
    const double nlo = (first == 0) ? lo : lo + w * (double)first / 33.0;
    const double nhi = (first == 32) ? hi : lo + w * (double)(first + 1) / 33.0;
    lo = nlo;
    hi = nhi;
  }
  const double lam = 0.5 * (lo + hi);
  // inverse iteration: (T - sigma I) y = rhs, sigma slightly below lambda,
  // with the tridiagonal LU factorization with partial pivoting (row i
  // exchanged with row i + 1 when the subdiagonal entry is the larger):
  // L unit lower bidiagonal (multipliers ml, exchange flags sw), U upper
  // with diagonal ud and two superdiagonals u1, u2
  if (lane == 0) {
    const double sigma = lam - 1e-13 * tnorm;
    double* ud = &A[0][0];
    double* u1 = &A[1][0];
    double* u2 = &A[2][0];
    double* ml = &A[3][0];
    int* sw = reinterpret_cast<int*>(&A[4][0]);
    for (int i = 0; i < m; ++i) {
      ud[i] = al[i] - sigma;
      u1[i] = i + 1 < m ? be[i] : 0.0;
      u2[i] = 0.0;
    }
    for (int i = 0; i + 1 < m; ++i) {
      const double sub = be[i];  // entry (i + 1, i) before elimination
      if (fabs(ud[i]) >= fabs(sub)) {
        sw[i] = 0;
        if (fabs(ud[i]) < pivmin) ud[i] = pivmin;
        const double f = sub / ud[i];
        ml[i] = f;
        ud[i + 1] -= f * u1[i];
      } else {
        // exchange rows i and i + 1: new row i = (sub, ud[i+1], u1[i+1]),
        // new row i + 1 = (ud[i], u1[i], 0) minus f times the new row i
        sw[i] = 1;
        const double f = ud[i] / sub;
        ml[i] = f;
        const double r_d = ud[i + 1], r_u = i + 2 < m ? u1[i + 1] : 0.0;
        const double o_u = u1[i];
        ud[i] = sub;
        u1[i] = r_d;
        u2[i] = r_u;
        ud[i + 1] = o_u - f * r_d;
        if (i + 2 < m) u1[i + 1] = -f * r_u;
      }
    }
    if (fabs(ud[m - 1]) < pivmin) ud[m - 1] = pivmin;
    for (int i = 0; i < m; ++i) y[i] = 1.0 + 0.01 * (double)((i * 7919) % 101);
    for (int it = 0; it < 3; ++it) {
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm += y[i] * y[i];
      nrm = sqrt(nrm);
      for (int i = 0; i < m; ++i) rhs[i] = y[i] / nrm;
      // L z = P rhs
      for (int i = 0; i + 1 < m; ++i) {
        if (sw[i]) {
          const double t = rhs[i];
          rhs[i] = rhs[i + 1];
          rhs[i + 1] = t - ml[i] * rhs[i];
        } else {
          rhs[i + 1] -= ml[i] * rhs[i];
        }
      }
      // U y = z
      for (int i = m - 1; i >= 0; --i) {
        double s = rhs[i];
        if (i + 1 < m) s -= u1[i] * y[i + 1];
        if (i + 2 < m) s -= u2[i] * y[i + 2];
        y[i] = s / ud[i];
      }
    }
    double nrm = 0.0;
    int imax = 0;
    for (int i = 0; i < m; ++i) {
      nrm += y[i] * y[i];
      if (fabs(y[i]) > fabs(y[imax])) imax = i;
    }
    nrm = sqrt(nrm);
    const double sg = (y[imax] < 0) ? -1.0 : 1.0;
    for (int i = 0; i < m; ++i) st->y[i] = sg * y[i] / nrm;
    st->energy = lam;
    if (energy_out) *energy_out = lam;
    if (iters_out) *iters_out = m;
  }
}

// out[n] = sum_{i<m} y[i] V[i, n] and partial squared norms (FP64: this
// norm normalises the result vector).  Same alignment as update_kernel.
template <typename T>
__global__ void __launch_bounds__(VT) combine_kernel(const T* __restrict__ V, ll ldv,
                                                     const LzState* st, T* __restrict__ out,
                                                     ll n, double* __restrict__ partial) {
  using V16 = vec16_t<T>;
  constexpr int E = 16 / sizeof(T);
  __shared__ double sh[32];
  __shared__ T yc[KMAX];
  const int m = st->m;
  for (int i = threadIdx.x; i < m; i += VT) yc[i] = (T)st->y[i];
  __syncthreads();
  const ll nq = n / E;
  double nacc = 0.0;
  for (ll q = blockIdx.x * (ll)VT + threadIdx.x; q < nq; q += (ll)gridDim.x * VT) {
    V16 v = {};
#pragma unroll 8
    for (int i = 0; i < m; ++i) axpy_acc(v, yc[i], reinterpret_cast<const V16*>(V + (ll)i * ldv)[q]);
    reinterpret_cast<V16*>(out)[q] = v;
    nacc = sq_acc_f64(v, nacc);
  }
  if (blockIdx.x == 0) {
    for (ll e = nq * E + threadIdx.x; e < n; e += VT) {
      T v = T(0);
      for (int i = 0; i < m; ++i) v = fma(yc[i], V[(ll)i * ldv + e], v);
      out[e] = v;
      nacc = fma((double)v, (double)v, nacc);
    }
  }
  double s = block_sum(nacc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// ---- Gram-Schmidt of the bf16x3 sweep: FP32 basis, double-FP32 arithmetic.
// The basis vectors are stored in FP32 (the operator products they feed
// carry ~2^-16 relative error).  The projections of the work vector on them,
// the work vector itself and the final combination are carried as
// unevaluated sums hi + lo of two floats (about 48 significant bits, the
// accuracy class of FP64), formed with error-free products (one FMA recovers
// the rounding error of a float product) and error-free two-sums (Dekker
// 1971; Knuth, TAOCP vol. 2, Sect. 4.2.2).  All of it runs on the FP32 units:
// on GB300 the FP64 units (including the float-to-double conversions) are
// too slow for one multiply-add per basis element at HBM speed.  The _rn
// intrinsics keep the compiler from contracting the error terms away.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// basis vectors loaded ahead of the double-FP32 update chains (bytes in flight)
constexpr int UB = 8;

// (ah, al) += (xh + xl) v
__device__ __forceinline__ void ff_mac(float& ah, float& al, float xh, float xl, float v) {
  const float p = __fmul_rn(xh, v);
  float e = __fmaf_rn(xh, v, -p);  // xh v - p exactly
  e = __fmaf_rn(xl, v, e);
  float s, t;
  two_sum_f(ah, p, s, t);
  ah = s;
  al = __fadd_rn(al, __fadd_rn(t, e));
}

// (xh, xl) -= (ch + cl) v
__device__ __forceinline__ void ff_sub(float& xh, float& xl, float ch, float cl, float v) {
  const float p = __fmul_rn(ch, v);
  float e = __fmaf_rn(ch, v, -p);
  e = __fmaf_rn(cl, v, e);
  float s, t;
  two_sum_f(xh, -p, s, t);
  xh = s;
  xl = __fadd_rn(xl, __fsub_rn(t, e));
}

// double-FP32 parts of an FP64 scalar
__device__ __forceinline__ void split_ff(double c, float& h, float& l) {
  h = (float)c;
  l = (float)(c - (double)h);
}

// partial[blk * ldp + i] = sum over this block's elements of V[i, n] x[n]
// with x = xh + xl (xl may be null: a fresh FP32 operator product); per
// thread in double-FP32, block sums in FP64; the pass structure of
// dots_kernel.
__global__ void __launch_bounds__(VT) dots_ff_kernel(const float* __restrict__ V, ll ldv, int nv,
                                                     const float* __restrict__ xh_, const float* __restrict__ xl_,
                                                     ll n, double* __restrict__ partial, int ldp, const int* stop) {
  if (stopped(stop)) return;
  __shared__ double sh[VT / 32][DV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const ll nq = n / 4;
  const int npass = (nv + DV - 1) / DV;
  const int per = (nv + npass - 1) / npass;
  for (int i0 = 0; i0 < nv; i0 += per) {
    const int cnt = nv - i0 < per ? nv - i0 : per;
    const float* Vb = V + (ll)i0 * ldv;
    float ah[DV], al[DV];
#pragma unroll
    for (int c = 0; c < DV; ++c) ah[c] = al[c] = 0.f;
    for (ll q = blockIdx.x * (ll)VT + threadIdx.x; q < nq; q += (ll)gridDim.x * VT) {
      const float4 xh = reinterpret_cast<const float4*>(xh_)[q];
      const float4 xl = xl_ ? reinterpret_cast<const float4*>(xl_)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int c = 0; c < DV; ++c) {
        if (c < cnt) {
          const float4 v = reinterpret_cast<const float4*>(Vb + (ll)c * ldv)[q];
          ff_mac(ah[c], al[c], xh.x, xl.x, v.x);
          ff_mac(ah[c], al[c], xh.y, xl.y, v.y);
          ff_mac(ah[c], al[c], xh.z, xl.z, v.z);
          ff_mac(ah[c], al[c], xh.w, xl.w, v.w);
        }
      }
    }
    if (blockIdx.x == 0) {
      for (ll e = nq * 4 + threadIdx.x; e < n; e += VT) {
        const float xh = xh_[e], xl = xl_ ? xl_[e] : 0.f;
#pragma unroll
        for (int c = 0; c < DV; ++c)
          if (c < cnt) ff_mac(ah[c], al[c], xh, xl, Vb[(ll)c * ldv + e]);
      }
    }
#pragma unroll
    for (int c = 0; c < DV; ++c) {
      if (c < cnt) {
        const double v = warp_sum((double)ah[c] + (double)al[c]);
        if (lane == 0) sh[warp][c] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < VT / 32; ++w) t += sh[w][threadIdx.x];
      partial[(ll)blockIdx.x * ldp + i0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// (oh, ol) = (xh + xl) - sum_i coef[i] V[i, n] in double-FP32 (xl may be
// null; out may be x); with want_norm the partial squared norm of the result
// (double-FP32 per thread, FP64 block sum).
__global__ void __launch_bounds__(VT) update_ff_kernel(const float* __restrict__ V, ll ldv, int nv,
                                                       const double* __restrict__ coef, const float* xh_,
                                                       const float* xl_, float* oh_, float* ol_, ll n,
                                                       int want_norm, double* __restrict__ partial, int ldp,
                                                       const int* stop) {
  if (stopped(stop)) return;
  __shared__ double sh[32];
  __shared__ float ch[KMAX], cl[KMAX];
  for (int i = threadIdx.x; i < nv; i += VT) split_ff(coef[i], ch[i], cl[i]);
  __syncthreads();
  const ll nq = n / 4;
  float nh = 0.f, nl = 0.f;
  for (ll q = blockIdx.x * (ll)VT + threadIdx.x; q < nq; q += (ll)gridDim.x * VT) {
    const float4 h4 = reinterpret_cast<const float4*>(xh_)[q];
    const float4 l4 = xl_ ? reinterpret_cast<const float4*>(xl_)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    float xh[4] = {h4.x, h4.y, h4.z, h4.w}, xl[4] = {l4.x, l4.y, l4.z, l4.w};
    for (int i0 = 0; i0 < nv; i0 += UB) {
      // UB basis loads in flight before their (sequential) subtractions
      float4 bb[UB];
#pragma unroll
      for (int u = 0; u < UB; ++u)
        bb[u] = i0 + u < nv ? reinterpret_cast<const float4*>(V + (ll)(i0 + u) * ldv)[q]
                            : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        if (i0 + u < nv) {
          const int i = i0 + u;
          ff_sub(xh[0], xl[0], ch[i], cl[i], bb[u].x);
          ff_sub(xh[1], xl[1], ch[i], cl[i], bb[u].y);
          ff_sub(xh[2], xl[2], ch[i], cl[i], bb[u].z);
          ff_sub(xh[3], xl[3], ch[i], cl[i], bb[u].w);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s, e;
      two_sum_f(xh[k], xl[k], s, e);  // renormalise: |lo| below half an ulp of hi
      xh[k] = s;
      xl[k] = e;
      ff_mac(nh, nl, xh[k], __fmul_rn(2.f, xl[k]), xh[k]);  // (h + l)^2 without l^2
    }
    reinterpret_cast<float4*>(oh_)[q] = make_float4(xh[0], xh[1], xh[2], xh[3]);
    reinterpret_cast<float4*>(ol_)[q] = make_float4(xl[0], xl[1], xl[2], xl[3]);
  }
  if (blockIdx.x == 0) {
    for (ll e = nq * 4 + threadIdx.x; e < n; e += VT) {
      float xh = xh_[e], xl = xl_ ? xl_[e] : 0.f;
      for (int i = 0; i < nv; ++i) ff_sub(xh, xl, ch[i], cl[i], V[(ll)i * ldv + e]);
      float s, t;
      two_sum_f(xh, xl, s, t);
      oh_[e] = s;
      ol_[e] = t;
      ff_mac(nh, nl, s, __fmul_rn(2.f, t), s);
    }
  }
  if (want_norm) {
    const double sum = block_sum((double)nh + (double)nl, sh);
    if (threadIdx.x == 0) partial[(ll)blockIdx.x * ldp] = sum;
  }
}

// First Gram-Schmidt pass and the projections of the second, in one sweep
// over the basis: (oh, ol) = x - sum_i coef[i] V[i, n] with x a fresh FP32
// operator product, and partial[blk * ldp + i] = sum over this block's
// elements of V[i, n] (oh + ol)[n], i < nv <= FV.  Each thread re-reads the
// basis elements it has just used (cache hits), so the basis streams from
// HBM once for both steps.  Arithmetic as in update_ff_kernel and
// dots_ff_kernel (double-FP32 per thread, block sums in FP64).
constexpr int FV = 24;  // largest basis of the fused pass

__global__ void __launch_bounds__(VT) update_dots_ff_kernel(const float* __restrict__ V, ll ldv, int nv,
                                                            const double* __restrict__ coef,
                                                            const float* __restrict__ x_, float* __restrict__ oh_,
                                                            float* __restrict__ ol_, ll n,
                                                            double* __restrict__ partial, int ldp,
                                                            const int* stop) {
  if (stopped(stop)) return;
  __shared__ double sh[VT / 32][FV];
  __shared__ float ch[FV], cl[FV];
  for (int i = threadIdx.x; i < nv; i += VT) split_ff(coef[i], ch[i], cl[i]);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float ah[FV], al[FV];
#pragma unroll
  for (int c = 0; c < FV; ++c) ah[c] = al[c] = 0.f;
  const ll nq = n / 4;
  for (ll q = blockIdx.x * (ll)VT + threadIdx.x; q < nq; q += (ll)gridDim.x * VT) {
    const float4 x4 = reinterpret_cast<const float4*>(x_)[q];
    float xh[4] = {x4.x, x4.y, x4.z, x4.w}, xl[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i0 = 0; i0 < nv; i0 += UB) {
      // UB basis loads in flight before their (sequential) subtractions
      float4 bb[UB];
#pragma unroll
      for (int u = 0; u < UB; ++u)
        bb[u] = i0 + u < nv ? reinterpret_cast<const float4*>(V + (ll)(i0 + u) * ldv)[q]
                            : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        if (i0 + u < nv) {
          const int i = i0 + u;
          ff_sub(xh[0], xl[0], ch[i], cl[i], bb[u].x);
          ff_sub(xh[1], xl[1], ch[i], cl[i], bb[u].y);
          ff_sub(xh[2], xl[2], ch[i], cl[i], bb[u].z);
          ff_sub(xh[3], xl[3], ch[i], cl[i], bb[u].w);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s, e;
      two_sum_f(xh[k], xl[k], s, e);
      xh[k] = s;
      xl[k] = e;
    }
    reinterpret_cast<float4*>(oh_)[q] = make_float4(xh[0], xh[1], xh[2], xh[3]);
    reinterpret_cast<float4*>(ol_)[q] = make_float4(xl[0], xl[1], xl[2], xl[3]);
#pragma unroll
    for (int c = 0; c < FV; ++c) {
      if (c < nv) {
        const float4 v = reinterpret_cast<const float4*>(V + (ll)c * ldv)[q];
        ff_mac(ah[c], al[c], xh[0], xl[0], v.x);
        ff_mac(ah[c], al[c], xh[1], xl[1], v.y);
        ff_mac(ah[c], al[c], xh[2], xl[2], v.z);
        ff_mac(ah[c], al[c], xh[3], xl[3], v.w);
      }
    }
  }
  if (blockIdx.x == 0) {
    for (ll e = nq * 4 + threadIdx.x; e < n; e += VT) {
      float xh = x_[e], xl = 0.f;
      for (int i = 0; i < nv; ++i) ff_sub(xh, xl, ch[i], cl[i], V[(ll)i * ldv + e]);
      float s, t;
      two_sum_f(xh, xl, s, t);
      oh_[e] = s;
      ol_[e] = t;
#pragma unroll
      for (int c = 0; c < FV; ++c)
        if (c < nv) ff_mac(ah[c], al[c], s, t, V[(ll)c * ldv + e]);
    }
  }
#pragma unroll
  for (int c = 0; c < FV; ++c) {
    if (c < nv) {
      const double v = warp_sum((double)ah[c] + (double)al[c]);
      if (lane == 0) sh[warp][c] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < VT / 32; ++w) t += sh[w][threadIdx.x];
    partial[(ll)blockIdx.x * ldp + threadIdx.x] = t;
  }
}

// v_out[n] = (xh + xl)[n] / sqrt(*norm2), rounded to FP32 (the next basis vector)
__global__ void normalize_ff_kernel(const float* __restrict__ xh, const float* __restrict__ xl,
                                    float* __restrict__ out, ll n, const double* norm2, const int* stop) {
  if (stopped(stop)) return;
  float sh, sl;
  split_ff(1.0 / sqrt(*norm2), sh, sl);
  for (ll e = blockIdx.x * (ll)VT + threadIdx.x; e < n; e += (ll)gridDim.x * VT) {
    const float h = xh[e], l = xl[e];
    out[e] = __fmaf_rn(h, sh, __fmaf_rn(l, sh, __fmul_rn(h, sl)));
  }
}

// (oh, ol)[n] = sum_i y_i V[i, n] in double-FP32 and its partial squared norm
__global__ void __launch_bounds__(VT) combine_ff_kernel(const float* __restrict__ V, ll ldv,
                                                        const LzState* st, float* __restrict__ oh_,
                                                        float* __restrict__ ol_, ll n,
                                                        double* __restrict__ partial) {
  __shared__ double sh[32];
  __shared__ float yh[KMAX], yl[KMAX];
  const int m = st->m;
  for (int i = threadIdx.x; i < m; i += VT) split_ff(-st->y[i], yh[i], yl[i]);  // ff_sub of -y adds y
  __syncthreads();
  const ll nq = n / 4;
  float nh = 0.f, nl = 0.f;
  for (ll q = blockIdx.x * (ll)VT + threadIdx.x; q < nq; q += (ll)gridDim.x * VT) {
    float xh[4] = {0.f, 0.f, 0.f, 0.f}, xl[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i0 = 0; i0 < m; i0 += UB) {
      float4 bb[UB];
#pragma unroll
      for (int u = 0; u < UB; ++u)
        bb[u] = i0 + u < m ? reinterpret_cast<const float4*>(V + (ll)(i0 + u) * ldv)[q]
                           : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        if (i0 + u < m) {
          const int i = i0 + u;
          ff_sub(xh[0], xl[0], yh[i], yl[i], bb[u].x);
          ff_sub(xh[1], xl[1], yh[i], yl[i], bb[u].y);
          ff_sub(xh[2], xl[2], yh[i], yl[i], bb[u].z);
          ff_sub(xh[3], xl[3], yh[i], yl[i], bb[u].w);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s, e;
      two_sum_f(xh[k], xl[k], s, e);
      xh[k] = s;
      xl[k] = e;
      ff_mac(nh, nl, xh[k], __fmul_rn(2.f, xl[k]), xh[k]);
    }
    reinterpret_cast<float4*>(oh_)[q] = make_float4(xh[0], xh[1], xh[2], xh[3]);
    reinterpret_cast<float4*>(ol_)[q] = make_float4(xl[0], xl[1], xl[2], xl[3]);
  }
  if (blockIdx.x == 0) {
    for (ll e = nq * 4 + threadIdx.x; e < n; e += VT) {
      float xh = 0.f, xl = 0.f;
      for (int i = 0; i < m; ++i) ff_sub(xh, xl, yh[i], yl[i], V[(ll)i * ldv + e]);
      float s, t;
      two_sum_f(xh, xl, s, t);
      oh_[e] = s;
      ol_[e] = t;
      ff_mac(nh, nl, s, __fmul_rn(2.f, t), s);
    }
  }
  const double sum = block_sum((double)nh + (double)nl, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = sum;
}

// theta[n] = (xh + xl)[n] / sqrt(*norm2) in FP64 (the Ritz vector)
__global__ void normalize_ff_to_f64_kernel(const float* __restrict__ xh, const float* __restrict__ xl,
                                           double* __restrict__ out, ll n, const double* norm2) {
  const double s = 1.0 / sqrt(*norm2);
  for (ll e = blockIdx.x * (ll)VT + threadIdx.x; e < n; e += (ll)gridDim.x * VT)
    out[e] = ((double)xh[e] + (double)xl[e]) * s;
}

// y = exp(tau T) e_1 / |exp(tau T) e_1| for the Lanczos tridiagonal T (m x m):
// T = Q Lambda Q^T by cyclic two-sided Jacobi on the dense m x m matrix in
// shared memory (one warp: each rotation's row and column updates are spread
// over the lanes), then y = Q exp(tau (Lambda - lambda_ref)) Q^T e_1 with
// lambda_ref the value of largest tau lambda (a common factor, removed by
// the normalisation).  alpha0 = T_00 = <v_0, H v_0>.
__global__ void tridiag_expm_kernel(LzState* st, double tau, double* alpha0, int* iters_out) {
  __shared__ double A[KMAX][KMAX + 1];
  __shared__ double Q[KMAX][KMAX + 1];
  const int lane = threadIdx.x;
  const int m = st->m;
  for (int i = lane; i < m; i += 32)
    for (int j = 0; j < m; ++j) {
      double a = 0.0;
      if (i == j) a = st->alpha[i];
      else if (j == i + 1) a = st->beta[i];
      else if (i == j + 1) a = st->beta[j];
      A[i][j] = a;
      Q[i][j] = (i == j) ? 1.0 : 0.0;
    }
  __syncwarp();
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int i = lane; i < m; i += 32) {
      dg += A[i][i] * A[i][i];
      for (int j = i + 1; j < m; ++j) off += A[i][j] * A[i][j];
    }
    off = warp_sum(off);
    dg = warp_sum(dg);
    if (!(off > 1e-32 * (dg + 1e-300))) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[p][q];
        if (apq == 0.0) continue;  // uniform: every lane reads the same entry
        const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        __syncwarp();
        for (int k = lane; k < m; k += 32) {  // columns p, q
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        __syncwarp();
        for (int k = lane; k < m; k += 32) {  // rows p, q
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
          const double qkp = Q[k][p], qkq = Q[k][q];
          Q[k][p] = c * qkp - s * qkq;
          Q[k][q] = s * qkp + c * qkq;
        }
        __syncwarp();
      }
  }
  // largest tau lambda
  double ref = -1e300;
  for (int i = 0; i < m; ++i) ref = fmax(ref, tau * A[i][i]);
  __shared__ double ysh[KMAX];
  double nrm = 0.0;
  for (int j = lane; j < m; j += 32) {
    double acc = 0.0;
    for (int i = 0; i < m; ++i) acc += Q[j][i] * exp(tau * A[i][i] - ref) * Q[0][i];
    ysh[j] = acc;
    nrm += acc * acc;
  }
  nrm = warp_sum(nrm);
  __syncwarp();
  const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
  for (int j = lane; j < m; j += 32) st->y[j] = ysh[j] * inv;
  if (lane == 0) {
    if (alpha0) *alpha0 = st->alpha[0];
    if (iters_out) *iters_out = m;
  }
}

__global__ void init_lz_kernel(LzState* st, int k, double tol) {
  if (threadIdx.x == 0) {
    st->m = 0;
    st->stop = 0;
    st->k = k;
    st->tol = tol;
  }
}

// ----------------------------------------------------------------- PCG
struct PcgState {
  double bnorm2, rnorm2, rz, rz_new, pAp, alpha, beta, rel;
  int iters, done, maxiter;
  double rtol;
};

__global__ void pcg_init_kernel(PcgState* st, int maxiter, double rtol) {
  if (threadIdx.x == 0) {
    st->iters = 0;
    st->done = 0;
    st->maxiter = maxiter;
    st->rtol = rtol;
    st->rel = 0.0;
  }
}

// r = b - Ax; z = P r; p = z   (elementwise)
__global__ void pcg_start_kernel(const double* __restrict__ b, const double* __restrict__ Ax,
                                 const double* __restrict__ diag, double* __restrict__ r,
                                 double* __restrict__ z, double* __restrict__ p, ll n) {
  for (ll e = blockIdx.x * (ll)VT + threadIdx.x; e < n; e += (ll)gridDim.x * VT) {
    double rv = b[e] - Ax[e];
    r[e] = rv;
    double zv = diag ? rv / diag[e] : rv;
    z[e] = zv;
    p[e] = zv;
  }
}

// partial sums of up to three products: (a0*b0, a1*b1, a2*b2)
__global__ void __launch_bounds__(VT) dot3_kernel(const double* a0, const double* b0,
                                                  const double* a1, const double* b1,
                                                  const double* a2, const double* b2, ll n,
                                                  double* __restrict__ partial, const int* stop) {
  if (stopped(stop)) return;
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (ll e = blockIdx.x * (ll)VT + threadIdx.x; e < n; e += (ll)gridDim.x * VT) {
    if (a0) s0 = fma(a0[e], b0[e], s0);
    if (a1) s1 = fma(a1[e], b1[e], s1);
    if (a2) s2 = fma(a2[e], b2[e], s2);
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 3 + 0] = s0;
    partial[blockIdx.x * 3 + 1] = s1;
    partial[blockIdx.x * 3 + 2] = s2;
  }
}

// after <b,b>, <r,r>, <r,z>: set up the scalars and decide whether r0 already meets rtol
__global__ void pcg_setup_kernel(PcgState* st, const double* sums) {
  if (threadIdx.x) return;
  st->bnorm2 = sums[0];
  st->rnorm2 = sums[1];
  st->rz = sums[2];
  st->rel = st->bnorm2 > 0 ? sqrt(st->rnorm2 / st->bnorm2) : 0.0;
  if (st->bnorm2 == 0.0 || st->rnorm2 <= st->rtol * st->rtol * st->bnorm2 || st->maxiter <= 0)
    st->done = 1;
}

__global__ void pcg_alpha_kernel(PcgState* st, const double* sums) {
  if (threadIdx.x || st->done) return;
  st->pAp = sums[0];
  st->alpha = st->rz / st->pAp;
  if (!(st->pAp > 0.0) || !isfinite(st->alpha)) st->done = 2;  // not SPD / breakdown
}

// x += alpha p; r -= alpha Ap; z = P r   (elementwise)
__global__ void pcg_update_kernel(const PcgState* st, double* __restrict__ x,
                                  double* __restrict__ r, double* __restrict__ z,
                                  const double* __restrict__ p, const double* __restrict__ Ap,
                                  const double* __restrict__ diag, ll n) {
  if (st->done) return;
  const double a = st->alpha;
  for (ll e = blockIdx.x * (ll)VT + threadIdx.x; e < n; e += (ll)gridDim.x * VT) {
    x[e] = fma(a, p[e], x[e]);
    double rv = fma(-a, Ap[e], r[e]);
    r[e] = rv;
    z[e] = diag ? rv / diag[e] : rv;
  }
}

// after <r,r>, <r,z>: convergence test and beta
__global__ void pcg_beta_kernel(PcgState* st, const double* sums) {
  if (threadIdx.x || st->done) return;
  st->iters += 1;
  st->rnorm2 = sums[0];
  st->rz_new = sums[1];
  st->rel = sqrt(st->rnorm2 / st->bnorm2);
  if (st->rnorm2 <= st->rtol * st->rtol * st->bnorm2 || st->iters >= st->maxiter) {
    st->done = 1;
    return;
  }
  st->beta = st->rz_new / st->rz;
  st->rz = st->rz_new;
}

// p = z + beta p
__global__ void pcg_dir_kernel(const PcgState* st, double* __restrict__ p,
                               const double* __restrict__ z, ll n) {
  if (st->done) return;
  const double b = st->beta;
  for (ll e = blockIdx.x * (ll)VT + threadIdx.x; e < n; e += (ll)gridDim.x * VT) p[e] = fma(b, p[e], z[e]);
}

__global__ void pcg_finish_kernel(const PcgState* st, double* resid_out, int* iters_out) {
  if (threadIdx.x) return;
  if (resid_out) *resid_out = st->rel;
  if (iters_out) *iters_out = st->iters;
}

int vec_grid(const seemps_ctx* ctx, ll n) { return stride_grid(ctx, n, VT, 8); }

// Resident blocks per SM of a kernel at VT threads (queried once per kernel).
template <typename K>
int resident_blocks(K kernel) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, VT, 0) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return b;
}

// One full wave of the kernel (resident blocks x SMs), fewer when the
// vectors have fewer 16-byte chunks than threads.
template <typename T>
int wave_grid(const seemps_ctx* ctx, int resident, ll n) {
  const ll chunks = (n + 16 / (ll)sizeof(T) - 1) / (16 / (ll)sizeof(T));
  ll want = (chunks + VT - 1) / VT;
  const ll cap = (ll)ctx->sm_count * resident;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

template <typename T>
struct VecGrids {
  int dots, update, combine;
  VecGrids(const seemps_ctx* ctx, ll n) {
    // queried once (thread-safe statics; the same device type for every context)
    static const int rd = resident_blocks(dots_kernel<T>);
    static const int ru = resident_blocks(update_kernel<T>);
    static const int rc = resident_blocks(combine_kernel<T>);
    dots = wave_grid<T>(ctx, rd, n);
    update = wave_grid<T>(ctx, ru, n);
    combine = wave_grid<T>(ctx, rc, n);
  }
  int max() const {
    int m = dots > update ? dots : update;
    return m > combine ? m : combine;
  }
};

}  // namespace

// ================================================================= Lanczos
size_t lanczos_workspace_bytes(int chi, int d, int D, int k) {
  const size_t n = (size_t)round_up((ll)chi * d * d * chi, 32);  // padded basis rows
  return (size_t)(k + 2) * n * 8 + heff_workspace_bytes(chi, d, D) + 64 * 1024 + 2048 * KMAX * 8;
}

// Lanczos on an already planned operator (the sweep reuses its plan).
// The Lanczos recurrence with full re-orthogonalisation (CGS2) from
// v_0 = theta / |theta|: basis V (k + 1 vectors of n, type T) and the
// tridiagonal (alpha, beta) in st; the work vector w and the block partials
// are returned for the finishers.
template <typename T>
struct LzRun {
  LzState* st;
  T *V, *w;
  float *wh, *wl;  // FP32 basis: the double-FP32 work vector of the Gram-Schmidt passes
  double* partial;
  ll ldv;
  int G, Gc;
};

// Grids of the FP64-arithmetic Gram-Schmidt kernels (one resident wave).
struct MixedGrids {
  int dots, upd, combine, fused;
  MixedGrids(const seemps_ctx* ctx, ll n) {
    static const int a = resident_blocks(dots_ff_kernel);
    static const int c = resident_blocks(update_ff_kernel);
    static const int e = resident_blocks(combine_ff_kernel);
    static const int f = resident_blocks(update_dots_ff_kernel);
    dots = wave_grid<float>(ctx, a, n);
    fused = wave_grid<float>(ctx, f, n);
    upd = wave_grid<float>(ctx, c, n);
    combine = wave_grid<float>(ctx, e, n);
  }
  int max() const {
    int m = dots > upd ? dots : upd;
    m = m > fused ? m : fused;
    return m > combine ? m : combine;
  }
};

template <typename T>
static seemps_status lanczos_build(seemps_ctx* ctx, const HeffPlan* plan, ll n, const double* theta, int k,
                                   double tol, LzRun<T>* r) {
  constexpr bool MIXED = std::is_same<T, float>::value;
  const int G = vec_grid(ctx, n);
  const VecGrids<T> vg(ctx, n);
  const int Gd = vg.dots, Gu = vg.update;
  const int Gt = VecGrids<double>(ctx, n).dots;
  int Gp = vg.max() > G ? vg.max() : G;
  Gp = Gp > Gt ? Gp : Gt;
  MixedGrids mg(ctx, MIXED ? n : 1);
  if (MIXED && mg.max() > Gp) Gp = mg.max();
  LzState* st;
  T *V, *w;
  float *wh = nullptr, *wl = nullptr;
  double* partial;
  const ll ldv = round_up(n, 32);  // 16-byte aligned rows
  SEEMPS_TRY(ws_alloc(ctx, 1, &st));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)(k + 1) * ldv, &V));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)ldv, &w));
  if (MIXED) {
    SEEMPS_TRY(ws_alloc(ctx, (size_t)ldv, &wh));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)ldv, &wl));
  }
  SEEMPS_TRY(ws_alloc(ctx, (size_t)Gp * KMAX, &partial));
  init_lz_kernel<<<1, 32, 0, ctx->stream>>>(st, k, tol);
  SEEMPS_LAUNCHED(ctx);
  // v_0 = theta / |theta|  (theta is the caller's pointer: scalar access)
  dots_kernel<double><<<Gt, VT, 0, ctx->stream>>>(theta, n, 1, theta, n, partial, KMAX, nullptr, 0);
  SEEMPS_LAUNCHED(ctx);
  reduce_kernel<<<1, 256, 0, ctx->stream>>>(partial, Gt, KMAX, 1, &st->norm2, nullptr);
  SEEMPS_LAUNCHED(ctx);
  normalize_kernel<double, T><<<G, VT, 0, ctx->stream>>>(theta, V, n, &st->norm2, nullptr);
  SEEMPS_LAUNCHED(ctx);
  const int* saved_skip = ctx->skip;
  ctx->skip = &st->stop;
  seemps_status rc = SEEMPS_OK;
  for (int j = 0; j < k && rc == SEEMPS_OK; ++j) {
    T* vj = V + (ll)j * ldv;
    rc = heff_run(ctx, plan, vj, w);
    if (rc != SEEMPS_OK) break;
    const int nv = j + 1;
    if constexpr (MIXED) {
      // FP32 product w; c1 = V^T w (FP32 products and per-thread sums, FP64
      // block sums: the second pass removes what this pass leaves);
      // (wh, wl) = w - V c1 ; c2 = V^T (wh + wl) ; (wh, wl) -= V c2 ;
      // |wh + wl|^2 -- these in double-FP32
      dots_kernel<float><<<Gd, VT, 0, ctx->stream>>>(V, ldv, nv, w, n, partial, KMAX, &st->stop, 1);
      reduce_kernel<<<nv, 256, 0, ctx->stream>>>(partial, Gd, KMAX, nv, st->c1, &st->stop);
      if (nv <= FV) {
        // the first update and the second pass's projections share one read of V
        update_dots_ff_kernel<<<mg.fused, VT, 0, ctx->stream>>>(V, ldv, nv, st->c1, w, wh, wl, n, partial, KMAX,
                                                                &st->stop);
        reduce_kernel<<<nv, 256, 0, ctx->stream>>>(partial, mg.fused, KMAX, nv, st->c2, &st->stop);
      } else {
        update_ff_kernel<<<mg.upd, VT, 0, ctx->stream>>>(V, ldv, nv, st->c1, w, nullptr, wh, wl, n, 0, partial,
                                                         KMAX, &st->stop);
        dots_ff_kernel<<<mg.dots, VT, 0, ctx->stream>>>(V, ldv, nv, wh, wl, n, partial, KMAX, &st->stop);
        reduce_kernel<<<nv, 256, 0, ctx->stream>>>(partial, mg.dots, KMAX, nv, st->c2, &st->stop);
      }
      update_ff_kernel<<<mg.upd, VT, 0, ctx->stream>>>(V, ldv, nv, st->c2, wh, wl, wh, wl, n, 1, partial,
                                                       KMAX, &st->stop);
      reduce_kernel<<<1, 256, 0, ctx->stream>>>(partial, mg.upd, KMAX, 1, &st->norm2, &st->stop);
      lz_control_kernel<<<1, 32, 0, ctx->stream>>>(st, j);
      normalize_ff_kernel<<<G, VT, 0, ctx->stream>>>(wh, wl, V + (ll)(j + 1) * ldv, n, &st->scale, &st->stop);
    } else {
      // c1 = V^T w ; w -= V c1
      dots_kernel<T><<<Gd, VT, 0, ctx->stream>>>(V, ldv, nv, w, n, partial, KMAX, &st->stop, 1);
      reduce_kernel<<<nv, 256, 0, ctx->stream>>>(partial, Gd, KMAX, nv, st->c1, &st->stop);
      update_kernel<T><<<Gu, VT, 0, ctx->stream>>>(V, ldv, nv, st->c1, w, n, 0, partial, KMAX, &st->stop);
      // c2 = V^T w ; w -= V c2 ; |w|^2
      dots_kernel<T><<<Gd, VT, 0, ctx->stream>>>(V, ldv, nv, w, n, partial, KMAX, &st->stop, 1);
      reduce_kernel<<<nv, 256, 0, ctx->stream>>>(partial, Gd, KMAX, nv, st->c2, &st->stop);
      update_kernel<T><<<Gu, VT, 0, ctx->stream>>>(V, ldv, nv, st->c2, w, n, 1, partial, KMAX, &st->stop);
      reduce_kernel<<<1, 256, 0, ctx->stream>>>(partial, Gu, KMAX, 1, &st->norm2, &st->stop);
      lz_control_kernel<<<1, 32, 0, ctx->stream>>>(st, j);
      normalize_kernel<T, T><<<G, VT, 0, ctx->stream>>>(w, V + (ll)(j + 1) * ldv, n, &st->scale, &st->stop);
    }
    ctx->launches += (MIXED && nv <= FV) ? 8 : 9;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      seemps_set_error(ctx, "lanczos launch: %s", cudaGetErrorString(e));
      rc = SEEMPS_ERR_CUDA;
    }
  }
  ctx->skip = saved_skip;
  SEEMPS_TRY(rc);
  r->st = st;
  r->V = V;
  r->w = w;
  r->wh = wh;
  r->wl = wl;
  r->partial = partial;
  r->ldv = ldv;
  r->G = G;
  r->Gc = MIXED ? mg.combine : vg.combine;
  return SEEMPS_OK;
}

// theta = the normalised combination sum_j y_j v_j of the basis (y in st)
template <typename T>
static seemps_status lanczos_combine(seemps_ctx* ctx, const LzRun<T>& r, ll n, double* theta) {
  if constexpr (std::is_same<T, float>::value) {
    combine_ff_kernel<<<r.Gc, VT, 0, ctx->stream>>>(r.V, r.ldv, r.st, r.wh, r.wl, n, r.partial);
    SEEMPS_LAUNCHED(ctx);
    reduce_kernel<<<1, 256, 0, ctx->stream>>>(r.partial, r.Gc, 1, 1, &r.st->norm2, nullptr);
    SEEMPS_LAUNCHED(ctx);
    normalize_ff_to_f64_kernel<<<r.G, VT, 0, ctx->stream>>>(r.wh, r.wl, theta, n, &r.st->norm2);
    SEEMPS_LAUNCHED(ctx);
    return SEEMPS_OK;
  }
  combine_kernel<T><<<r.Gc, VT, 0, ctx->stream>>>(r.V, r.ldv, r.st, r.w, n, r.partial);
  SEEMPS_LAUNCHED(ctx);
  reduce_kernel<<<1, 256, 0, ctx->stream>>>(r.partial, r.Gc, 1, 1, &r.st->norm2, nullptr);
  SEEMPS_LAUNCHED(ctx);
  normalize_kernel<T, double><<<r.G, VT, 0, ctx->stream>>>(r.w, theta, n, &r.st->norm2, nullptr);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

// Lowest eigenpair (finish = 0) or Krylov exponential (finish = 1) with a
// basis of type T.
template <typename T>
static seemps_status krylov_local(seemps_ctx* ctx, const HeffPlan* plan, ll n, double* theta, int k, double tol,
                                  int finish, double tau, double* value_out, int* iters_out) {
  LzRun<T> r;
  SEEMPS_TRY(lanczos_build<T>(ctx, plan, n, theta, k, tol, &r));
  if (finish == 0) tridiag_lowest_kernel<<<1, 32, 0, ctx->stream>>>(r.st, value_out, iters_out);
  else tridiag_expm_kernel<<<1, 32, 0, ctx->stream>>>(r.st, tau, value_out, iters_out);
  SEEMPS_LAUNCHED(ctx);
  return lanczos_combine<T>(ctx, r, n, theta);
}

seemps_status lanczos_run(seemps_ctx* ctx, const HeffPlan* plan, ll n, double* theta, int k,
                          double tol, double* energy_out, int* iters_out) {
  SEEMPS_REQUIRE(ctx, k >= 1 && k <= KMAX, "local_eig: krylov_dim must be in [1, %d]", KMAX);
  if ((ll)k > n) k = (int)n;
  PhaseTimer timer(ctx, SEEMPS_PHASE_LOCAL);
  if (plan->precision == SEEMPS_BF16X3)
    return krylov_local<float>(ctx, plan, n, theta, k, tol, 0, 0.0, energy_out, iters_out);
  return krylov_local<double>(ctx, plan, n, theta, k, tol, 0, 0.0, energy_out, iters_out);
}

seemps_status expm_run(seemps_ctx* ctx, const HeffPlan* plan, ll n, double* theta, int k, double tol,
                       double tau, double* alpha0, int* iters_out) {
  SEEMPS_REQUIRE(ctx, k >= 1 && k <= KMAX, "local_expm: krylov_dim must be in [1, %d]", KMAX);
  if ((ll)k > n) k = (int)n;
  PhaseTimer timer(ctx, SEEMPS_PHASE_LOCAL);
  if (plan->precision == SEEMPS_BF16X3)
    return krylov_local<float>(ctx, plan, n, theta, k, tol, 1, tau, alpha0, iters_out);
  return krylov_local<double>(ctx, plan, n, theta, k, tol, 1, tau, alpha0, iters_out);
}

extern "C" seemps_status seemps_local_expm(seemps_ctx* ctx, const seemps_pair_dims* dims, int sites,
                                           const double* L, const double* W1, const double* W2,
                                           const double* R, double* theta_inout, int krylov_dim,
                                           double breakdown_tol, double tau, int precision, double* alpha0_out,
                                           int* iters_out) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, dims && theta_inout, "local_expm: null argument");
  SEEMPS_REQUIRE(ctx, sites == 1 || sites == 2, "local_expm: sites must be 1 or 2");
  WsFrame frame(ctx);
  HeffPlan plan;
  if (sites == 2) SEEMPS_TRY(heff_plan(ctx, dims, L, W1, W2, R, precision, &plan));
  else SEEMPS_TRY(heff1_plan(ctx, dims, L, W1, R, precision, &plan));
  const ll n = (ll)dims->chi_l * plan.dp * dims->chi_r;
  return expm_run(ctx, &plan, n, theta_inout, krylov_dim, breakdown_tol, tau, alpha0_out, iters_out);
}

extern "C" seemps_status seemps_local_eig(seemps_ctx* ctx, const seemps_pair_dims* dims,
                                          const double* L, const double* W1, const double* W2,
                                          const double* R, double* theta_inout, int krylov_dim,
                                          double breakdown_tol, int precision, double* energy_out,
                                          int* iters_out) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, dims && theta_inout, "local_eig: null argument");
  WsFrame frame(ctx);
  HeffPlan planv;
  HeffPlan* plan = &planv;
  SEEMPS_TRY(heff_plan(ctx, dims, L, W1, W2, R, precision, plan));
  const ll n = (ll)dims->chi_l * dims->d * dims->d * dims->chi_r;
  return lanczos_run(ctx, plan, n, theta_inout, krylov_dim, breakdown_tol, energy_out, iters_out);
}

// ================================================================= PCG
size_t pcg_workspace_bytes(int chi, int d, int D) {
  const size_t n = (size_t)chi * d * d * chi;
  return 6 * n * 8 + heff_workspace_bytes(chi, d, D) + 64 * 1024;
}

// Preconditioner hooks: z = P r for the learned preconditioner (mlp.cu).
size_t mlp_state_bytes();
seemps_status mlp_precond_prepare(seemps_ctx* ctx, const seemps_mlp* mlp, const seemps_pair_dims* dm,
                                  int site, int n_sites, const double* L, const double* R,
                                  const double* diag, void* storage);
seemps_status mlp_precond_apply(seemps_ctx* ctx, void* storage, const double* r, double* z,
                                const int* skip);

seemps_status pcg_run(seemps_ctx* ctx, const HeffPlan* plan, const seemps_pair_dims* dm,
                      const double* L, const double* W1, const double* W2, const double* R,
                      const double* b, double* x, int precond, const seemps_mlp* mlp, int site,
                      int n_sites, double rtol, int maxiter, double* resid_out, int* iters_out) {
  const ll n = (ll)dm->chi_l * dm->d * dm->d * dm->chi_r;
  PhaseTimer timer(ctx, SEEMPS_PHASE_LOCAL);
  const int G = vec_grid(ctx, n);
  PcgState* st;
  double *r, *z, *p, *Ap, *diag = nullptr, *partial, *sums;
  SEEMPS_TRY(ws_alloc(ctx, 1, &st));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n, &r));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n, &z));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n, &p));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)n, &Ap));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)G * 3, &partial));
  SEEMPS_TRY(ws_alloc(ctx, 4, &sums));
  void* mstate = nullptr;
  alignas(16) char mstate_buf[256];
  if (precond == SEEMPS_PRECOND_JACOBI || precond == SEEMPS_PRECOND_MLP) {
    SEEMPS_TRY(ws_alloc(ctx, (size_t)n, &diag));
    SEEMPS_TRY(seemps_heff_diagonal(ctx, dm, L, W1, W2, R, diag));
  }
  if (precond == SEEMPS_PRECOND_MLP) {
    SEEMPS_REQUIRE(ctx, mlp != nullptr, "local_pcg: MLP preconditioner without a network");
    SEEMPS_REQUIRE(ctx, mlp_state_bytes() <= sizeof(mstate_buf), "internal: MLP state size");
    SEEMPS_TRY(mlp_precond_prepare(ctx, mlp, dm, site, n_sites, L, R, diag, mstate_buf));
    mstate = mstate_buf;
  }
  const double* dj = (precond == SEEMPS_PRECOND_JACOBI) ? diag : nullptr;
  pcg_init_kernel<<<1, 32, 0, ctx->stream>>>(st, maxiter, rtol);
  SEEMPS_LAUNCHED(ctx);
  SEEMPS_TRY(heff_run(ctx, plan, x, Ap));
  pcg_start_kernel<<<G, VT, 0, ctx->stream>>>(b, Ap, dj, r, z, p, n);
  SEEMPS_LAUNCHED(ctx);
  if (mstate) {
    SEEMPS_TRY(mlp_precond_apply(ctx, mstate, r, z, nullptr));
    SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(p, z, n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  dot3_kernel<<<G, VT, 0, ctx->stream>>>(b, b, r, r, r, z, n, partial, nullptr);
  SEEMPS_LAUNCHED(ctx);
  reduce_kernel<<<3, 256, 0, ctx->stream>>>(partial, G, 3, 3, sums, nullptr);
  SEEMPS_LAUNCHED(ctx);
  pcg_setup_kernel<<<1, 32, 0, ctx->stream>>>(st, sums);
  SEEMPS_LAUNCHED(ctx);
  const int* saved_skip = ctx->skip;
  ctx->skip = &st->done;
  seemps_status rc = SEEMPS_OK;
  int hdone = 0;
  for (int it = 0; it < maxiter && rc == SEEMPS_OK; ++it) {
    rc = heff_run(ctx, plan, p, Ap);
    if (rc != SEEMPS_OK) break;
    dot3_kernel<<<G, VT, 0, ctx->stream>>>(p, Ap, nullptr, nullptr, nullptr, nullptr, n, partial,
                                            &st->done);
    reduce_kernel<<<1, 256, 0, ctx->stream>>>(partial, G, 3, 1, sums, &st->done);
    pcg_alpha_kernel<<<1, 32, 0, ctx->stream>>>(st, sums);
    pcg_update_kernel<<<G, VT, 0, ctx->stream>>>(st, x, r, z, p, Ap, dj, n);
    ctx->launches += 4;
    if (mstate) rc = mlp_precond_apply(ctx, mstate, r, z, &st->done);
    if (rc != SEEMPS_OK) break;
    dot3_kernel<<<G, VT, 0, ctx->stream>>>(r, r, r, z, nullptr, nullptr, n, partial, &st->done);
    reduce_kernel<<<2, 256, 0, ctx->stream>>>(partial, G, 3, 2, sums, &st->done);
    pcg_beta_kernel<<<1, 32, 0, ctx->stream>>>(st, sums);
    pcg_dir_kernel<<<G, VT, 0, ctx->stream>>>(st, p, z, n);
    ctx->launches += 4;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      seemps_set_error(ctx, "pcg launch: %s", cudaGetErrorString(e));
      rc = SEEMPS_ERR_CUDA;
      break;
    }
    // every 8 iterations, look at the done flag on the host so that a solve
    // that converged early does not queue hundreds of no-op launches
    if ((it & 7) == 7) {
      cudaError_t e1 = cudaMemcpyAsync(ctx->h_status, &st->done, sizeof(int),
                                       cudaMemcpyDeviceToHost, ctx->stream);
      cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
      if (e1 != cudaSuccess || e2 != cudaSuccess) {
        seemps_set_error(ctx, "pcg sync: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
        rc = SEEMPS_ERR_CUDA;
        break;
      }
      hdone = *ctx->h_status;
      *ctx->h_status = 0;
      if (hdone) break;
    }
  }
  ctx->skip = saved_skip;
  SEEMPS_TRY(rc);
  pcg_finish_kernel<<<1, 32, 0, ctx->stream>>>(st, resid_out, iters_out);
  SEEMPS_LAUNCHED(ctx);
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_local_pcg(seemps_ctx* ctx, const seemps_pair_dims* dims,
                                          const double* L, const double* W1, const double* W2,
                                          const double* R, const double* b, double* x_inout,
                                          int precond, const seemps_mlp* mlp, double rtol,
                                          int maxiter, int precision, double* resid_out,
                                          int* iters_out) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, dims && b && x_inout, "local_pcg: null argument");
  SEEMPS_REQUIRE(ctx, precond >= SEEMPS_PRECOND_NONE && precond <= SEEMPS_PRECOND_MLP,
                 "local_pcg: unknown preconditioner");
  SEEMPS_REQUIRE(ctx, maxiter >= 0, "local_pcg: negative maxiter");
  WsFrame frame(ctx);
  HeffPlan planv;
  HeffPlan* plan = &planv;
  SEEMPS_TRY(heff_plan(ctx, dims, L, W1, W2, R, precision, plan));
  return pcg_run(ctx, plan, dims, L, W1, W2, R, b, x_inout, precond, mlp, -1, 0, rtol, maxiter,
                 resid_out, iters_out);
}
