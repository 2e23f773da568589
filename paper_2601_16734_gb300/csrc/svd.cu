// Truncated SVD split of the two-site vector (Sect. 2.3): one-sided Jacobi
// (Hestenes), the truncation rank in FP64, and the re-layout of the kept
// factors into the new site tensors.
//
// FP64 path (svd_run<double>, also FP32 for small mixed-precision problems):
// the p = min(m, n) columns of X (X = M if n <= m, else X = M^T) are
// orthogonalised by plane rotations applied from the right; the same
// rotations accumulate in Q (p x p, starting at the identity).  Each column j
// of the stacked matrix G = [X; Q] is stored contiguously (length len + p,
// len = max(m, n)).  At convergence X = U S (columns orthogonal), so
// s_j = |X_j|, and M = U S Q^T (n <= m) or M = Q S U^T (n > m).  Pairs follow
// the round-robin (circle) schedule: p' - 1 steps of p'/2 disjoint pairs cover
// every pair once per sweep (p' = p rounded up to even).  A pair is rotated
// when |x_a . x_b| > tol |x_a| |x_b| with tol = max(4 eps, 2 sqrt(len) eps);
// a sweep without rotations ends the iteration.  Small problems (p <= 128)
// run every sweep inside one CTA (one warp per pair); larger ones inside one
// cooperative launch (one CTA per pair, a bounded grid barrier per step).
//
// Mixed-precision path for large problems (svd_noq_run): FP32 QR
// preconditioning, block-cyclic FP32 Jacobi on the isometric side only
// (svd_block_kernel) and the other factor by one tensor-core GEMM.
#include <math.h>

#include <utility>
#include <vector>

#include "common.cuh"
#include "timing.cuh"

namespace {

template <typename T> struct Eps;
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };

__device__ __forceinline__ double wsum(double v) { return warp_sum(v); }
__device__ __forceinline__ float wsum(float v) { return warp_sum_f(v); }

// Grid-wide barrier for a cooperative launch, bounded: a block that waits
// longer than `limit` SM clocks (the context's wait limit) gives up and
// reports failure.
__device__ bool grid_barrier(unsigned* arrive, unsigned* gen, unsigned nblk, long long limit) {
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
        if (clock64() - t0 > limit) {
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
                                                            int* sweeps_out, int* status, long long limit) {
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
          const T u = __ldcg(xa + i), v = __ldcg(xb + i);  // L2: other SMs rotated these
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
            const T u = __ldcg(xa + i), v = __ldcg(xb + i);
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
      if (!grid_barrier(bar, bar + 1, nblk, limit)) {
        if (threadIdx.x == 0) post_status(status, SEEMPS_ERR_TIMEOUT);
        return;
      }
    }
    if (*(volatile int*)(counts + sweep) == 0) break;  // same value in every block after the barrier
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = sweep;
}

// ------------------------------------------------------------------ block Jacobi
// Block-cyclic variant of the FP32 one-sided Jacobi.  The p columns form
// nb = ceil(p / B) blocks of B adjacent columns; blocks follow the
// round-robin schedule (nbp - 1 block steps of nbp / 2 disjoint block pairs,
// nbp = nb rounded up to even) and one CTA works on one block pair at a time.
// The CTA holds the 2B columns of its pair in registers, distributed by rows
// (thread t owns rows R t .. R t + R - 1 of every column), so a column pair
// needs no data movement: each thread forms its partial dot products, the
// warps reduce them and exchange one value per pair through shared memory
// (one CTA barrier per slot), and every warp then derives the rotations
// itself: lane c (c < 2B, mirrored in lanes 2B..31) carries column c's
// squared norm, scale and last change, and computes the rotation of the pair
// that holds column c.  A block step is a sequence of slots of B disjoint
// column pairs: at the first step of a sweep the B - 1 round-robin slots
// inside each block (both blocks at once), then B slots that pair column k of
// the first block with column (k + s) mod B of the second.  Every column pair
// is thus visited exactly once per sweep, at the same (step, slot) position.
//
// Rotations are applied in scaled form: the registers hold x~ with the
// column x = d x~, and the rotation x' = c x - s y, y' = s x + c y with
// t = s / c becomes x~' = x~ - (t d_y / d_x) y~, y~' = y~ + (t d_x / d_y) x~,
// d' = c d (two packed FMAs per element pair).  Scales are folded into the
// data before a block is written back.  c is renormalised so that
// c^2 (1 + t^2) = 1 up to its final rounding (error-free products).
//
// Column norms |x|^2 are recomputed from the data at the first step of every
// sweep and updated as a' = a - t g, b' = b + t g after a rotation.  A pair
// is skipped when neither column has changed since the pair's previous visit
// one sweep earlier (its outcome then cannot differ); a block step whose two
// blocks are unchanged since that time is skipped without touching the data.
// Blocks carry a 64-bit word (block steps completed | 1 + last change of any
// of its columns) handed between CTAs with release/acquire; one bounded grid
// barrier per sweep collects the rotation count.
constexpr int BJ_NT = 256;            // threads per CTA
constexpr int BJ_NW = BJ_NT / 32;     // warps per CTA
// words of the cleanup phase state (see svd_cleanup_kernel)
enum { CL_EN = 0, CL_FROM, CL_NS, CL_NC, CL_NR, CL_ST, CL_ROUNDS, CL_ROT, CL_VIS, CL_WORDS };

// Column pair k of slot s: inside the blocks (intra) or across them.
__host__ __device__ constexpr int bj_rr_a(int B, int s, int kk) {
  return kk == 0 ? s : (s + kk) % (B - 1);
}
__host__ __device__ constexpr int bj_rr_b(int B, int s, int kk) {
  return kk == 0 ? B - 1 : (s - kk + (B - 1)) % (B - 1);
}
__host__ __device__ constexpr int bj_pair_x(int B, bool intra, int s, int k) {
  return intra ? (k / (B / 2)) * B +
                     (bj_rr_a(B, s, k % (B / 2)) < bj_rr_b(B, s, k % (B / 2)) ? bj_rr_a(B, s, k % (B / 2))
                                                                              : bj_rr_b(B, s, k % (B / 2)))
               : k;
}
__host__ __device__ constexpr int bj_pair_y(int B, bool intra, int s, int k) {
  return intra ? (k / (B / 2)) * B +
                     (bj_rr_a(B, s, k % (B / 2)) < bj_rr_b(B, s, k % (B / 2)) ? bj_rr_b(B, s, k % (B / 2))
                                                                              : bj_rr_a(B, s, k % (B / 2)))
               : B + (k + s) % B;
}

// Tangent t and cosine c of the Jacobi rotation that zeroes the dot product
// g of two columns with squared norms ax, ay:
//   t = sign(u) 2g / (|u| + sqrt(u^2 + 4g^2)),  u = ay - ax  (sign(0) = 1),
// (the smaller root of t^2 + (u/g) t - 1 = 0, without forming u/g), and
// c = 1/sqrt(1 + t^2) corrected once so that c^2 (1 + t^2) - 1, evaluated
// with error-free products, vanishes.  Needs u^2 + 4g^2 within FP32 range.
__device__ __forceinline__ void bj_rotation(float ax, float ay, float g, float* t_out, float* c_out) {
  const float u = ay - ax, w = 2.f * g;
  const float q = fmaf(u, u, w * w);
  const float t = __fdividef(u >= 0.f ? w : -w, fabsf(u) + q * rsqrtf(q));
  float c = rsqrtf(fmaf(t, t, 1.f));
  const float c2h = c * c, c2l = fmaf(c, c, -c2h);
  const float t2h = t * t, t2l = fmaf(t, t, -t2h);
  const float r = fmaf(c2h, t2h, c2h - 1.f) + fmaf(c2l, 1.f + t2h, c2h * t2l);
  c = fmaf(-0.5f * r, c, c);
  *t_out = t;
  *c_out = c;
}

// Per-warp state of the block pair: lane l describes column l & 15.
struct BjCol {
  float alpha;  // squared norm of the column
  float dsc;    // scale: column = dsc * registers
  int lm;       // slot time of the column's last rotation (-1: never)
};

template <int B>
struct BjRed {
  float v[2][BJ_NW][B];  // per-warp partial dot products, double buffered by slot
};

// One slot of B column pairs.  `stale` marks columns unchanged since before
// the previous visit, `mod` the columns rotated in this block step; both are
// uniform across the CTA.
template <int B, int R, bool INTRA, int S>
__device__ __forceinline__ void bj_slot(float2 (&v)[2 * B][R / 2], BjRed<B>& red, int& buf, BjCol& col,
                                        unsigned present, unsigned& stale, unsigned& mod, int& nrot,
                                        int& nvis, int t_slot, float tol, int lane, int warp) {
  constexpr unsigned M = (1u << B) - 1u;
  unsigned act = 0;
  if constexpr (!INTRA) {
    // pair k = (k, B + (k + S) mod B): rotate the second block's bits right by S
    const unsigned pJ = (present >> B) & M, sJ = (stale >> B) & M;
    const unsigned pJr = S == 0 ? pJ : (((pJ >> S) | (pJ << (B - S))) & M);
    const unsigned sJr = S == 0 ? sJ : (((sJ >> S) | (sJ << (B - S))) & M);
    act = (present & M) & pJr & ~((stale & M) & sJr);
  } else {
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int x = bj_pair_x(B, INTRA, S, k), y = bj_pair_y(B, INTRA, S, k);
      const bool on = ((present >> x) & (present >> y) & 1u) && !((stale >> x) & (stale >> y) & 1u);
      act |= (on ? 1u : 0u) << k;
    }
  }
  if (act == 0) return;  // uniform: nothing to do in this slot
  nvis += __popc(act);
  float part[B];
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const int x = bj_pair_x(B, INTRA, S, k), y = bj_pair_y(B, INTRA, S, k);
    float2 acc = make_float2(0.f, 0.f);
    if ((act >> k) & 1u) {
#pragma unroll
      for (int r = 0; r < R / 2; ++r) acc = __ffma2_rn(v[x][r], v[y][r], acc);
    }
    part[k] = acc.x + acc.y;
  }
  const float tot = rs_reduce<B>(part, lane);
  if (lane < B) red.v[buf][warp][rs_index<B>(lane)] = tot;
  __syncthreads();
  // the pair and partner of this lane's column
  const int c = lane & 15;
  int kc = -1, pc = c;
  bool isx = false;
  if constexpr (!INTRA) {
    if (c < B) {
      kc = c;
      pc = B + ((c + S) & (B - 1));
      isx = true;
    } else if (c < 2 * B) {
      kc = (c - B + B - S) & (B - 1);
      pc = kc;
    }
  } else {
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int x = bj_pair_x(B, INTRA, S, k), y = bj_pair_y(B, INTRA, S, k);
      if (c == x) { kc = k; pc = y; isx = true; }
      if (c == y) { kc = k; pc = x; isx = false; }
    }
  }
  const bool kact = kc >= 0 && ((act >> kc) & 1u);
  float g = 0.f;
  if (kact) {
#pragma unroll
    for (int w = 0; w < BJ_NW; ++w) g += red.v[buf][w][kc];
  }
  const float a_p = __shfl_sync(0xffffffffu, col.alpha, pc);
  const float d_p = __shfl_sync(0xffffffffu, col.dsc, pc);
  float mult = 0.f;
  bool did = false;
  if (kact) {
    const float ax = isx ? col.alpha : a_p, ay = isx ? a_p : col.alpha;
    const float dx = isx ? col.dsc : d_p, dy = isx ? d_p : col.dsc;
    const float G = dx * dy * g;
    if (G != 0.f && fabsf(G) * rsqrtf(ax) * rsqrtf(ay) > tol) {
      float t, cr;
      bj_rotation(ax, ay, G, &t, &cr);
      did = true;
      if (isx) {
        mult = __fdividef(t * dy, dx);
        col.alpha = fmaxf(fmaf(-t, G, col.alpha), 0.f);
      } else {
        mult = __fdividef(t * dx, dy);
        col.alpha = fmaxf(fmaf(t, G, col.alpha), 0.f);
      }
      col.dsc *= cr;
      col.lm = t_slot;
    }
  }
  const unsigned rm = __ballot_sync(0xffffffffu, did) & 0xffffu;  // rotated columns
  if (rm) {
    mod |= rm;
    stale &= ~rm;
    nrot += __popc(rm) >> 1;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int x = bj_pair_x(B, INTRA, S, k), y = bj_pair_y(B, INTRA, S, k);
      if ((rm >> x) & 1u) {
        // volatile shuffles keep the pairs' multipliers from being fetched
        // all at once (register pressure)
        float mx, my;
        asm volatile("shfl.sync.idx.b32 %0, %1, %2, 31, -1;" : "=f"(mx) : "f"(mult), "r"(x));
        asm volatile("shfl.sync.idx.b32 %0, %1, %2, 31, -1;" : "=f"(my) : "f"(mult), "r"(y));
        const float2 nmx = make_float2(-mx, -mx), pmy = make_float2(my, my);
#pragma unroll
        for (int r = 0; r < R / 2; ++r) {
          const float2 xo = v[x][r];
          v[x][r] = __ffma2_rn(nmx, v[y][r], xo);
          v[y][r] = __ffma2_rn(pmy, xo, v[y][r]);
        }
      }
    }
  }
  buf ^= 1;
}

template <int B, int R, bool INTRA, int... S>
__device__ __forceinline__ void bj_slots(std::integer_sequence<int, S...>, float2 (&v)[2 * B][R / 2],
                                         BjRed<B>& red, int& buf, BjCol& col, unsigned present,
                                         unsigned& stale, unsigned& mod, int& nrot, int& nvis, int t0,
                                         float tol, int lane, int warp) {
  (bj_slot<B, R, INTRA, S>(v, red, buf, col, present, stale, mod, nrot, nvis, t0 + S, tol, lane, warp), ...);
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <int B, int R>
__global__ void __launch_bounds__(BJ_NT, 1) svd_block_kernel(
    float* __restrict__ X, int p, int len, int nb, int nbp, float tol, int max_sweeps,
    int* __restrict__ counts, unsigned* bar, int* sweeps_out, int* status, float* __restrict__ nrm,
    int* __restrict__ lm, unsigned long long* __restrict__ blk, long long limit, int switch_rot, int* cl) {
  constexpr int C = 2 * B;
  constexpr int TS = 2 * B - 1;  // slots per block step (intra slots only used at step 0)
  static_assert(C <= 16 && (B & (B - 1)) == 0 && B >= 2 && R % 2 == 0, "block shape");
  __shared__ BjRed<B> red;
  __shared__ float red16[BJ_NW][16];
  __shared__ int mode_s;
  __shared__ unsigned blk_s[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int period = (nbp - 1) * TS;
  const unsigned nblk = gridDim.x;
  volatile int* vabort = reinterpret_cast<volatile int*>(bar + 2);
  const bool vec = (len % 4 == 0);
  float2 v[C][R / 2];
  int buf = 0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int nrot = 0, nvis = 0;
    for (int step = 0; step < nbp - 1; ++step) {
      const int g = sweep * (nbp - 1) + step;
      const int tp0 = g * TS - period;  // time of this step's first slot one sweep earlier
      for (int kp = blockIdx.x; kp < nbp / 2; kp += nblk) {
        int I, J;
        rr_pair(step, kp, nbp, &I, &J);
        if (I > J) { const int q = I; I = J; J = q; }
        if (tid == 0) {
          int ok = 1;
          unsigned long long wI = 0, wJ = 0;
          const long long t0 = clock64();
          for (;;) {
            wI = ld_acquire64(blk + I);
            wJ = ld_acquire64(blk + J);
            if ((int)(unsigned)wI >= g && (int)(unsigned)wJ >= g) break;
            if (*vabort != 0) { ok = 0; break; }
            if (clock64() - t0 > limit) {
              post_status(status, SEEMPS_ERR_TIMEOUT);
              *vabort = 1;
              ok = 0;
              break;
            }
            __nanosleep(32);
          }
          // high word: 1 + last change of any column of the block (0: never)
          const int mI = (int)(wI >> 32) - 1, mJ = (int)(wJ >> 32) - 1;
          int mode = ok ? 2 : 0;  // 0: abandon, 1: unchanged pair of blocks, 2: work
          if (ok && sweep > 0 && mI < tp0 && mJ < tp0) mode = 1;
          mode_s = mode;
          blk_s[0] = (unsigned)(wI >> 32);
          blk_s[1] = (unsigned)(wJ >> 32);
        }
        __syncthreads();
        const int mode = mode_s;
        if (mode == 2) {
          // columns: data rows R tid .. R tid + R - 1; lane scalars of column lane & 15
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int bk = c < B ? I : J;
            const int cc = bk * B + (c % B);
            const bool pres = bk < nb && cc < p;
            const float* src = X + (ll)cc * len + (ll)R * tid;
            bool done = false;
            if constexpr (R % 4 == 0) {
              if (pres && vec && R * tid + R <= len) {
#pragma unroll
                for (int r = 0; r < R / 2; r += 2) {
                  const float4 q4 = __ldcg(reinterpret_cast<const float4*>(src + 2 * r));
                  v[c][r] = make_float2(q4.x, q4.y);
                  v[c][r + 1] = make_float2(q4.z, q4.w);
                }
                done = true;
              }
            }
            if (!done) {
#pragma unroll
              for (int r = 0; r < R / 2; ++r) {
                const int i0 = R * tid + 2 * r;
                v[c][r] = make_float2(pres && i0 < len ? __ldcg(src + 2 * r) : 0.f,
                                      pres && i0 + 1 < len ? __ldcg(src + 2 * r + 1) : 0.f);
              }
            }
          }
          const int c = lane & 15;
          const int cbk = c < B ? I : J;
          const int ccol = cbk * B + (c % B);
          const bool cpres = c < C && cbk < nb && ccol < p;
          BjCol col;
          col.lm = cpres ? __ldcg(lm + ccol) : -1;
          col.alpha = cpres ? __ldcg(nrm + ccol) : 0.f;
          col.dsc = 1.f;
          const unsigned present = __ballot_sync(0xffffffffu, cpres) & 0xffffu;
          unsigned stale = __ballot_sync(0xffffffffu, cpres && sweep > 0 && col.lm < tp0) & 0xffffu;
          unsigned mod = 0;
          if (step == 0) {
            // exact norms at the start of every sweep (two groups of B columns)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float part[B];
#pragma unroll
              for (int q = 0; q < B; ++q) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < R / 2; ++r) acc = __ffma2_rn(v[h * B + q][r], v[h * B + q][r], acc);
                part[q] = acc.x + acc.y;
              }
              const float tot = rs_reduce<B>(part, lane);
              if (lane < B) red16[warp][h * B + rs_index<B>(lane)] = tot;
            }
            __syncthreads();
            float a = 0.f;
#pragma unroll
            for (int w = 0; w < BJ_NW; ++w) a += red16[w][c];
            if (cpres) col.alpha = a;
            bj_slots<B, R, true>(std::make_integer_sequence<int, B - 1>{}, v, red, buf, col, present, stale,
                                 mod, nrot, nvis, g * TS, tol, lane, warp);
          }
          bj_slots<B, R, false>(std::make_integer_sequence<int, B>{}, v, red, buf, col, present, stale, mod,
                                nrot, nvis, g * TS + (B - 1), tol, lane, warp);
          // fold the scales into the rotated columns and write them back; the
          // block indices pass through an opaque move so that the column
          // addresses are formed here rather than kept live from the loads
          int Io, Jo;
          asm volatile("mov.b32 %0, %1;" : "=r"(Io) : "r"(I));
          asm volatile("mov.b32 %0, %1;" : "=r"(Jo) : "r"(J));
#pragma unroll
          for (int q = 0; q < C; ++q) {
            if ((mod >> q) & 1u) {
              const float dq = __shfl_sync(0xffffffffu, col.dsc, q);
              const float2 d2 = make_float2(dq, dq);
              const int bk = q < B ? Io : Jo;
              const int cc = bk * B + (q % B);
              float* dst = X + (ll)cc * len + (ll)R * tid;
#pragma unroll
              for (int r = 0; r < R / 2; ++r) v[q][r] = __fmul2_rn(v[q][r], d2);
              if (R * tid < len) {
                bool done = false;
                if constexpr (R % 4 == 0) {
                  if (vec && R * tid + R <= len) {
#pragma unroll
                    for (int r = 0; r < R / 2; r += 2)
                      __stcg(reinterpret_cast<float4*>(dst + 2 * r),
                             make_float4(v[q][r].x, v[q][r].y, v[q][r + 1].x, v[q][r + 1].y));
                    done = true;
                  }
                }
                if (!done) {
#pragma unroll
                  for (int r = 0; r < R / 2; ++r) {
                    const int i0 = R * tid + 2 * r;
                    if (i0 < len) __stcg(dst + 2 * r, v[q][r].x);
                    if (i0 + 1 < len) __stcg(dst + 2 * r + 1, v[q][r].y);
                  }
                }
              }
            }
          }
          if (warp == 0) {
            if (lane < C && cpres && (step == 0 || ((mod >> c) & 1u))) {
              nrm[ccol] = col.alpha;
              lm[ccol] = col.lm;
            }
            int mI = (lane < B && cpres) ? col.lm : -1;
            int mJ = (lane >= B && lane < C && cpres) ? col.lm : -1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              mI = max(mI, __shfl_xor_sync(0xffffffffu, mI, o));
              mJ = max(mJ, __shfl_xor_sync(0xffffffffu, mJ, o));
            }
            if (lane == 0) {
              blk_s[0] = (unsigned)(mI + 1);
              blk_s[1] = (unsigned)(mJ + 1);
            }
          }
        }
        __syncthreads();  // the CTA's writes precede the release of the blocks
        if (tid == 0 && mode != 0) {
          st_release64(blk + I, ((unsigned long long)blk_s[0] << 32) | (unsigned)(g + 1));
          st_release64(blk + J, ((unsigned long long)blk_s[1] << 32) | (unsigned)(g + 1));
        }
      }
    }
    if (tid == 0) {
      if (nrot) atomicAdd(counts + sweep, nrot);
      if (nvis) atomicAdd(counts + max_sweeps + sweep, nvis);
    }
    if (!grid_barrier(bar, bar + 1, nblk, limit)) {
      if (tid == 0) post_status(status, SEEMPS_ERR_TIMEOUT);
      return;
    }
    if (*vabort != 0) return;
    const int rot = *(volatile int*)(counts + sweep);
    if (rot == 0) break;
    if (rot <= switch_rot && sweep + 1 < max_sweeps) {
      // few rotations left: the cleanup kernel finishes from the columns
      // rotated in this sweep (slot times >= sweep * period)
      if (blockIdx.x == 0 && tid == 0) {
        cl[CL_EN] = 1;
        cl[CL_FROM] = sweep * period;
      }
      ++sweep;
      break;
    }
  }
  if (blockIdx.x == 0 && tid == 0) *sweeps_out = sweep;
}

// ------------------------------------------------------------------ stationary blocks
// svd_block_kernel moves both blocks of every pair through L2 at every block
// step.  When the block count nbp is a power of two and every block pair
// has a CTA of its own (nbp / 2 CTAs), this variant orders the pairs so that
// one block of each pair stays in the CTA's registers for many steps: level
// h = 0, 1, ... of a sweep splits the blocks into groups of G = nbp / 2^h;
// the first half of a group is stationary (CTA j of the group keeps block
// base + j) and the second half circulates (at level step u, CTA j meets
// block base + G/2 + (j + u) mod G/2, handed on from CTA j + 1).  Level h
// pairs the halves of every group once, so the levels together (G/2 steps
// each, nbp - 1 in all) pair every two blocks exactly once per sweep, as the
// round-robin schedule does; only the circulating block is loaded and
// stored at a step, and a stationary block is written back when its CTA's
// stationary block changes (at level boundaries) and at the end.  Slots,
// rotations, the skip rules and the hand-off words are those of
// svd_block_kernel.
__device__ __forceinline__ void sm_pair(int k, int step, int nbp, int* S, int* M) {
  int half = nbp >> 1;
  while (half > 1 && step >= nbp - half) half >>= 1;
  const int u = step - (nbp - 2 * half);
  const int j = k % half, base = (k / half) * 2 * half;
  *S = base + j;
  *M = base + half + (j + u) % half;
}

// Columns h B .. h B + B - 1 of the register array from block bk.
template <int B, int R>
__device__ __forceinline__ void sm_load(float2 (&v)[2 * B][R / 2], int h, int bk, const float* __restrict__ X,
                                        int p, int nb, int len, bool vec, int tid) {
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const int cc = bk * B + q;
    const bool pres = bk < nb && cc < p;
    const float* src = X + (ll)cc * len + (ll)R * tid;
    bool done = false;
    if constexpr (R % 4 == 0) {
      if (pres && vec && R * tid + R <= len) {
#pragma unroll
        for (int r = 0; r < R / 2; r += 2) {
          const float4 q4 = __ldcg(reinterpret_cast<const float4*>(src + 2 * r));
          v[h * B + q][r] = make_float2(q4.x, q4.y);
          v[h * B + q][r + 1] = make_float2(q4.z, q4.w);
        }
        done = true;
      }
    }
    if (!done) {
#pragma unroll
      for (int r = 0; r < R / 2; ++r) {
        const int i0 = R * tid + 2 * r;
        v[h * B + q][r] = make_float2(pres && i0 < len ? __ldcg(src + 2 * r) : 0.f,
                                      pres && i0 + 1 < len ? __ldcg(src + 2 * r + 1) : 0.f);
      }
    }
  }
}

// Store the columns h B + q of block bk whose bit q is set in `which`
// (scales already folded into the registers).
template <int B, int R>
__device__ __forceinline__ void sm_store(float2 (&v)[2 * B][R / 2], int h, int bk, unsigned which,
                                         float* __restrict__ X, int len, bool vec, int tid) {
#pragma unroll
  for (int q = 0; q < B; ++q) {
    if ((which >> q) & 1u) {
      float* dst = X + (ll)(bk * B + q) * len + (ll)R * tid;
      if (R * tid < len) {
        bool done = false;
        if constexpr (R % 4 == 0) {
          if (vec && R * tid + R <= len) {
#pragma unroll
            for (int r = 0; r < R / 2; r += 2)
              __stcg(reinterpret_cast<float4*>(dst + 2 * r),
                     make_float4(v[h * B + q][r].x, v[h * B + q][r].y, v[h * B + q][r + 1].x,
                                 v[h * B + q][r + 1].y));
            done = true;
          }
        }
        if (!done) {
#pragma unroll
          for (int r = 0; r < R / 2; ++r) {
            const int i0 = R * tid + 2 * r;
            if (i0 < len) __stcg(dst + 2 * r, v[h * B + q][r].x);
            if (i0 + 1 < len) __stcg(dst + 2 * r + 1, v[h * B + q][r].y);
          }
        }
      }
    }
  }
}

template <int B, int R>
__global__ void __launch_bounds__(BJ_NT, 1) svd_sm_kernel(
    float* __restrict__ X, int p, int len, int nb, int nbp, float tol, int max_sweeps,
    int* __restrict__ counts, unsigned* bar, int* sweeps_out, int* status, float* __restrict__ nrm,
    int* __restrict__ lm, unsigned long long* __restrict__ blk, long long limit, int switch_rot, int* cl) {
  constexpr int C = 2 * B;
  constexpr int TS = 2 * B - 1;
  constexpr unsigned LOW = (1u << B) - 1u;
  static_assert(C <= 16 && (B & (B - 1)) == 0 && B >= 2 && R % 2 == 0, "block shape");
  __shared__ BjRed<B> red;
  __shared__ float red16[BJ_NW][16];
  __shared__ int mode_s;
  __shared__ unsigned mark_s[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int period = (nbp - 1) * TS;
  const unsigned nblk = gridDim.x;
  const int k = blockIdx.x;  // this CTA's pair slot (gridDim.x == nbp / 2)
  volatile int* vabort = reinterpret_cast<volatile int*>(bar + 2);
  const bool vec = (len % 4 == 0);
  const int c = lane & 15;  // this lane's column of the pair (lanes 16-31 mirror 0-15)
  float2 v[C][R / 2];
  int buf = 0;
  int sweep = 0;
  int curS = -1;       // stationary block (its columns in v[0 .. B)), uniform
  bool haveS = false;  // its columns are loaded, uniform
  unsigned markS = 0;  // 1 + last change of any of its columns (0: never), uniform
  unsigned dirtyS = 0; // its columns changed since they were loaded, uniform
  BjCol col;
  col.alpha = 0.f;
  col.dsc = 1.f;
  col.lm = -1;
  // write the stationary block back and hand it on with step count g
  auto release_stationary = [&](int g) {
    if (curS < 0) return;
    if (haveS) {
      sm_store<B, R>(v, 0, curS, dirtyS, X, len, vec, tid);
      const int ccol = curS * B + c;
      if (warp == 0 && lane < B && curS < nb && ccol < p) {
        nrm[ccol] = col.alpha;
        lm[ccol] = col.lm;
      }
    }
    __syncthreads();  // the CTA's writes precede the release
    if (tid == 0) st_release64(blk + curS, ((unsigned long long)markS << 32) | (unsigned)g);
    haveS = false;
    dirtyS = 0;
  };
  for (; sweep < max_sweeps; ++sweep) {
    int nrot = 0, nvis = 0;
    for (int step = 0; step < nbp - 1; ++step) {
      const int g = sweep * (nbp - 1) + step;
      const int tp0 = g * TS - period;
      int S, M;
      sm_pair(k, step, nbp, &S, &M);
      bool needS = false;
      if (S != curS) {
        release_stationary(g);
        curS = S;
        needS = true;
      }
      if (tid == 0) {
        int ok = 1;
        unsigned long long wS = 0, wM = 0;
        const long long t0 = clock64();
        for (;;) {
          wM = ld_acquire64(blk + M);
          if (needS) wS = ld_acquire64(blk + S);
          if ((int)(unsigned)wM >= g && (!needS || (int)(unsigned)wS >= g)) break;
          if (*vabort != 0) { ok = 0; break; }
          if (clock64() - t0 > limit) {
            post_status(status, SEEMPS_ERR_TIMEOUT);
            *vabort = 1;
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
        const unsigned mS = needS ? (unsigned)(wS >> 32) : markS;
        const unsigned mM = (unsigned)(wM >> 32);
        int mode = ok ? 2 : 0;  // 0: abandon, 1: unchanged pair of blocks, 2: work
        if (ok && sweep > 0 && (int)mS - 1 < tp0 && (int)mM - 1 < tp0) mode = 1;
        mode_s = mode;
        mark_s[0] = mS;
        mark_s[1] = mM;
      }
      __syncthreads();
      const int mode = mode_s;
      markS = mark_s[0];
      unsigned markM = mark_s[1];
      if (mode == 2) {
        if (!haveS) {
          sm_load<B, R>(v, 0, S, X, p, nb, len, vec, tid);
          const int ccol = S * B + c;
          const bool pres = c < B && S < nb && ccol < p;
          if (c < B) {
            col.lm = pres ? __ldcg(lm + ccol) : -1;
            col.alpha = pres ? __ldcg(nrm + ccol) : 0.f;
            col.dsc = 1.f;
          }
          haveS = true;
          dirtyS = 0;
        }
        sm_load<B, R>(v, 1, M, X, p, nb, len, vec, tid);
        const int cbk = c < B ? S : M;
        const int ccol = cbk * B + (c % B);
        const bool cpres = c < C && cbk < nb && ccol < p;
        if (c >= B) {
          col.lm = cpres ? __ldcg(lm + ccol) : -1;
          col.alpha = cpres ? __ldcg(nrm + ccol) : 0.f;
          col.dsc = 1.f;
        }
        const unsigned present = __ballot_sync(0xffffffffu, cpres) & 0xffffu;
        unsigned stale = __ballot_sync(0xffffffffu, cpres && sweep > 0 && col.lm < tp0) & 0xffffu;
        unsigned mod = 0;
        if (step == 0) {
          // exact norms at the start of every sweep (two groups of B columns)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float part[B];
#pragma unroll
            for (int q = 0; q < B; ++q) {
              float2 acc = make_float2(0.f, 0.f);
#pragma unroll
              for (int r = 0; r < R / 2; ++r) acc = __ffma2_rn(v[h * B + q][r], v[h * B + q][r], acc);
              part[q] = acc.x + acc.y;
            }
            const float tot = rs_reduce<B>(part, lane);
            if (lane < B) red16[warp][h * B + rs_index<B>(lane)] = tot;
          }
          __syncthreads();
          float a = 0.f;
#pragma unroll
          for (int w = 0; w < BJ_NW; ++w) a += red16[w][c];
          if (cpres) col.alpha = a;
          bj_slots<B, R, true>(std::make_integer_sequence<int, B - 1>{}, v, red, buf, col, present, stale, mod,
                               nrot, nvis, g * TS, tol, lane, warp);
        }
        bj_slots<B, R, false>(std::make_integer_sequence<int, B>{}, v, red, buf, col, present, stale, mod, nrot,
                              nvis, g * TS + (B - 1), tol, lane, warp);
        // fold the scales of the rotated columns into the registers
#pragma unroll
        for (int q = 0; q < C; ++q) {
          if ((mod >> q) & 1u) {
            const float dq = __shfl_sync(0xffffffffu, col.dsc, q);
            const float2 d2 = make_float2(dq, dq);
#pragma unroll
            for (int r = 0; r < R / 2; ++r) v[q][r] = __fmul2_rn(v[q][r], d2);
          }
        }
        col.dsc = 1.f;
        dirtyS |= mod & LOW;
        // the circulating block goes back to memory; the stationary one stays
        int Mo;
        asm volatile("mov.b32 %0, %1;" : "=r"(Mo) : "r"(M));
        sm_store<B, R>(v, 1, Mo, (mod >> B) & LOW, X, len, vec, tid);
        if (warp == 0) {
          if (lane >= B && lane < C && cpres && (step == 0 || ((mod >> c) & 1u))) {
            nrm[ccol] = col.alpha;
            lm[ccol] = col.lm;
          }
          int mI = (lane < B && cpres) ? col.lm : -1;
          int mJ = (lane >= B && lane < C && cpres) ? col.lm : -1;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            mI = max(mI, __shfl_xor_sync(0xffffffffu, mI, o));
            mJ = max(mJ, __shfl_xor_sync(0xffffffffu, mJ, o));
          }
          if (lane == 0) {
            mark_s[0] = (unsigned)(mI + 1);
            mark_s[1] = (unsigned)(mJ + 1);
          }
        }
      }
      __syncthreads();  // the CTA's writes precede the release of the block
      if (mode == 2) {
        markS = mark_s[0];
        markM = mark_s[1];
      }
      if (tid == 0 && mode != 0) st_release64(blk + M, ((unsigned long long)markM << 32) | (unsigned)(g + 1));
      __syncthreads();  // mark_s is rewritten at the next step
    }
    if (tid == 0) {
      if (nrot) atomicAdd(counts + sweep, nrot);
      if (nvis) atomicAdd(counts + max_sweeps + sweep, nvis);
    }
    if (!grid_barrier(bar, bar + 1, nblk, limit)) {
      if (tid == 0) post_status(status, SEEMPS_ERR_TIMEOUT);
      return;
    }
    if (*vabort != 0) return;
    const int rot = *(volatile int*)(counts + sweep);
    if (rot == 0) break;
    if (rot <= switch_rot && sweep + 1 < max_sweeps) {
      if (blockIdx.x == 0 && tid == 0) {
        cl[CL_EN] = 1;
        cl[CL_FROM] = sweep * period;
      }
      ++sweep;
      break;
    }
  }
  // the stationary block's columns, norms and change times back to memory
  release_stationary((sweep < max_sweeps ? sweep : max_sweeps) * (nbp - 1));
  if (blockIdx.x == 0 && tid == 0) *sweeps_out = sweep;
}

// ------------------------------------------------------------------ cleanup
// The last block sweeps rotate few pairs yet cost nearly a full sweep each
// (every block step with one changed column still moves its blocks).  After
// a sweep with at most `switch_rot` rotations only the pairs that involve a
// column rotated in that sweep can still exceed the threshold (the others
// were checked in the sweep and neither column changed since).  The cleanup
// checks exactly those: with S the changed columns, it forms x_s . x_j for
// s in S and every j (FP32, each pair once), sorts the violating pairs by
// (s, j), rotates a maximal set of disjoint ones (greedy in that order: every
// violating pair keeps a rotated column, so it is checked again) and repeats
// with S = the rotated columns until no pair exceeds the threshold.  The
// stopping rule is the block sweep's: every pair within tol.
//
// State in cl[] (ints): CL_EN set by the block kernel when it hands over,
// CL_FROM the slot time at which that sweep began (lm >= CL_FROM: changed),
// CL_NS |S|, CL_NC candidates found, CL_NR rotations this round, CL_ST
// status (0 converged, 1 candidate overflow or round limit: more sweeps
// needed), CL_ROUNDS, CL_ROT total rotations, CL_VIS pairs checked.
constexpr int CL_CAP = 4096;   // violating pairs per round
constexpr int CL_MAXR = 48;    // rounds
constexpr int CL_CHUNK = 8;    // changed columns per work item

struct CleanupBuf {
  int* cl;      // CL_WORDS
  int* S;       // p: the changed columns (ascending)
  int* mark;    // p: 1 for columns in S
  int* ci;      // CL_CAP candidate pairs (i in S, j)
  int* cj;
  float* cg;    // their dot products and squared norms
  float* ca;
  float* cb;
  int* ri;      // p / 2 rotations of the round
  int* rj;
  float* rt;    // t and c of each rotation
  float* rc;
};

template <int R, int JB>
__global__ void __launch_bounds__(BJ_NT, 1) svd_cleanup_kernel(float* __restrict__ X, int p, int len, float tol,
                                                               CleanupBuf cb, const int* __restrict__ lm,
                                                               int* __restrict__ counts, const int* sweeps_out,
                                                               int max_sweeps, unsigned* bar, int* status,
                                                               long long limit) {
  __shared__ float redw[BJ_NW][CL_CHUNK * JB + JB];
  __shared__ float tot[CL_CHUNK * JB + JB];
  __shared__ float sa[CL_CHUNK];
  __shared__ int scol[CL_CHUNK];
  __shared__ unsigned long long keys[CL_CAP];
  __shared__ unsigned used[128];
  __shared__ int mlist[CL_CAP / 2];  // list indices of the chosen pairs (at most p / 2 <= 2048)
  __shared__ int s_n, s_nr;
  int* cl = cb.cl;
  // uniform: the block sweeps converged by themselves, or gave up on a wait
  if (cl[CL_EN] == 0 || *(volatile unsigned*)(bar + 2) != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned nblk = gridDim.x;
  // S from the last sweep's changes, in ascending column order (block 0)
  if (blockIdx.x == 0) {
    if (tid == 0) s_n = 0;
    __syncthreads();
    const int from = cl[CL_FROM];
    for (int c0 = 0; c0 < p; c0 += BJ_NT) {
      const int c = c0 + tid;
      const bool in = c < p && lm[c] >= from;
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      __shared__ int wbase[BJ_NW];
      if (lane == 0) wbase[warp] = __popc(bal);
      __syncthreads();
      if (tid == 0) {
        int run = s_n;
        for (int w = 0; w < BJ_NW; ++w) {
          const int k = wbase[w];
          wbase[w] = run;
          run += k;
        }
        s_n = run;
      }
      __syncthreads();
      if (in) cb.S[wbase[warp] + __popc(bal & ((1u << lane) - 1u))] = c;
      __syncthreads();
    }
    __syncthreads();
    for (int c = tid; c < p; c += BJ_NT) cb.mark[c] = 0;
    __syncthreads();
    for (int k = tid; k < s_n; k += BJ_NT) cb.mark[cb.S[k]] = 1;
    if (tid == 0) {
      cl[CL_NS] = s_n;
      cl[CL_NC] = 0;
      cl[CL_ST] = 0;
    }
  }
  if (!grid_barrier(bar, bar + 1, nblk, limit)) {
    if (tid == 0) post_status(status, SEEMPS_ERR_TIMEOUT);
    return;
  }
  int rounds = 0;
  for (; rounds < CL_MAXR; ++rounds) {
    const int ns = *(volatile int*)(cl + CL_NS);
    if (ns == 0) break;
    // ---- A: x_s . x_j for s in S, all j; violations to the candidate list
    const int nchunk = (ns + CL_CHUNK - 1) / CL_CHUNK;
    int jr = (int)nblk / nchunk;
    if (jr < 1) jr = 1;
    const int jlen = (p + jr - 1) / jr;
    int vis = 0;
    for (int item = blockIdx.x; item < nchunk * jr; item += nblk) {
      const int ch = item / jr, r0 = (item % jr) * jlen;
      const int r1 = r0 + jlen < p ? r0 + jlen : p;
      float v[CL_CHUNK][R];
      if (tid < CL_CHUNK) {
        const int k = ch * CL_CHUNK + tid;
        scol[tid] = k < ns ? cb.S[k] : -1;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < CL_CHUNK; ++q) {
        const int c = scol[q];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int i = R * tid + r;
          v[q][r] = (c >= 0 && i < len) ? __ldcg(X + (ll)c * len + i) : 0.f;
        }
      }
      {
        float part[CL_CHUNK];
#pragma unroll
        for (int q = 0; q < CL_CHUNK; ++q) {
          float acc = 0.f;
#pragma unroll
          for (int r = 0; r < R; ++r) acc = fmaf(v[q][r], v[q][r], acc);
          part[q] = acc;
        }
        const float t = rs_reduce<CL_CHUNK>(part, lane);
        if (lane < CL_CHUNK) redw[warp][rs_index<CL_CHUNK>(lane)] = t;
        __syncthreads();
        if (tid < CL_CHUNK) {
          float a = 0.f;
#pragma unroll
          for (int w = 0; w < BJ_NW; ++w) a += redw[w][tid];
          sa[tid] = a;
        }
        __syncthreads();
      }
      for (int j0 = r0; j0 < r1; j0 += JB) {
        float xj[JB][R];
#pragma unroll
        for (int b = 0; b < JB; ++b) {
          const int j = j0 + b;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int i = R * tid + r;
            xj[b][r] = (j < r1 && i < len) ? __ldcg(X + (ll)j * len + i) : 0.f;
          }
        }
        float part[CL_CHUNK * JB];
#pragma unroll
        for (int b = 0; b < JB; ++b)
#pragma unroll
          for (int q = 0; q < CL_CHUNK; ++q) {
            float acc = 0.f;
#pragma unroll
            for (int r = 0; r < R; ++r) acc = fmaf(v[q][r], xj[b][r], acc);
            part[b * CL_CHUNK + q] = acc;
          }
        float nj[JB];
#pragma unroll
        for (int b = 0; b < JB; ++b) {
          float acc = 0.f;
#pragma unroll
          for (int r = 0; r < R; ++r) acc = fmaf(xj[b][r], xj[b][r], acc);
          nj[b] = acc;
        }
        const float t = rs_reduce<CL_CHUNK * JB>(part, lane);
        const float tn = rs_reduce<JB>(nj, lane);
        if (lane < CL_CHUNK * JB) redw[warp][rs_index<CL_CHUNK * JB>(lane)] = t;
        if (lane < JB) redw[warp][CL_CHUNK * JB + rs_index<JB>(lane)] = tn;
        __syncthreads();
        if (tid < CL_CHUNK * JB + JB) {
          float a = 0.f;
#pragma unroll
          for (int w = 0; w < BJ_NW; ++w) a += redw[w][tid];
          tot[tid] = a;
        }
        __syncthreads();
        if (tid < CL_CHUNK * JB) {
          const int b = tid / CL_CHUNK, q = tid % CL_CHUNK;
          const int j = j0 + b, c = scol[q];
          // each pair once: (s, j) with j outside S, or both in S and s < j
          if (c >= 0 && j < r1 && j != c && (cb.mark[j] == 0 || c < j)) {
            ++vis;
            const float g = tot[tid], ax = sa[q], ay = tot[CL_CHUNK * JB + b];
            if (g != 0.f && fabsf(g) * rsqrtf(ax) * rsqrtf(ay) > tol) {
              const int k = atomicAdd(cl + CL_NC, 1);
              if (k < CL_CAP) {
                cb.ci[k] = c;
                cb.cj[k] = j;
                cb.cg[k] = g;
                cb.ca[k] = ax;
                cb.cb[k] = ay;
              }
            }
          }
        }
        __syncthreads();
      }
    }
    if (vis) atomicAdd(cl + CL_VIS, vis);
    if (!grid_barrier(bar, bar + 1, nblk, limit)) {
      if (tid == 0) post_status(status, SEEMPS_ERR_TIMEOUT);
      return;
    }
    // ---- B (block 0): sort the candidates by (s, j), greedy disjoint set, rotations
    if (blockIdx.x == 0) {
      const int ncand = *(volatile int*)(cl + CL_NC);
      const int nc = ncand < CL_CAP ? ncand : CL_CAP;
      int np2 = 1;
      while (np2 < nc) np2 <<= 1;
      for (int k = tid; k < np2; k += BJ_NT)
        keys[k] = k < nc ? (((unsigned long long)((ll)cb.ci[k] * p + cb.cj[k])) << 12) | (unsigned)k : ~0ULL;
      for (int w = tid; w < 128; w += BJ_NT) used[w] = 0u;
      __syncthreads();
      for (int size = 2; size <= np2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
          for (int k = tid; k < np2; k += BJ_NT) {
            const int l = k ^ stride;
            if (l > k) {
              const bool asc = (k & size) == 0;
              const unsigned long long a = keys[k], b = keys[l];
              if ((a > b) == asc) {
                keys[k] = b;
                keys[l] = a;
              }
            }
          }
          __syncthreads();
        }
      if (tid == 0) {
        // greedy in key order; the key carries the pair (s p + j) above the list index
        int nr = 0;
        for (int k = 0; k < nc; ++k) {
          const unsigned long long ij = keys[k] >> 12;
          const int i = (int)(ij / (unsigned)p), j = (int)(ij - (unsigned long long)i * p);
          const bool ui = (used[i >> 5] >> (i & 31)) & 1u, uj = (used[j >> 5] >> (j & 31)) & 1u;
          if (ui || uj) continue;
          used[i >> 5] |= 1u << (i & 31);
          used[j >> 5] |= 1u << (j & 31);
          mlist[nr++] = (int)(keys[k] & 0xFFFu);
        }
        s_nr = nr;
        cl[CL_NR] = nr;
        cl[CL_ROT] += nr;
        if (ncand > CL_CAP) cl[CL_ST] = 1;  // pairs were dropped: the caller runs more sweeps
      }
      __syncthreads();
      const int nr = s_nr;
      for (int k = tid; k < nr; k += BJ_NT) {
        const int e = mlist[k];
        float t, c;
        bj_rotation(cb.ca[e], cb.cb[e], cb.cg[e], &t, &c);
        cb.ri[k] = cb.ci[e];
        cb.rj[k] = cb.cj[e];
        cb.rt[k] = t;
        cb.rc[k] = c;
      }
      // next S: the rotated columns, ascending
      if (tid == 0) s_n = 0;
      __syncthreads();
      for (int c0 = 0; c0 < p; c0 += BJ_NT) {
        const int c = c0 + tid;
        const bool in = c < p && ((used[c >> 5] >> (c & 31)) & 1u);
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        __shared__ int wb2[BJ_NW];
        if (lane == 0) wb2[warp] = __popc(bal);
        __syncthreads();
        if (tid == 0) {
          int run = s_n;
          for (int w = 0; w < BJ_NW; ++w) {
            const int k = wb2[w];
            wb2[w] = run;
            run += k;
          }
          s_n = run;
        }
        __syncthreads();
        if (in) cb.S[wb2[warp] + __popc(bal & ((1u << lane) - 1u))] = c;
        if (c < p) cb.mark[c] = in ? 1 : 0;
        __syncthreads();
      }
      if (tid == 0) {
        cl[CL_NS] = cl[CL_ST] ? 0 : (nr ? s_n : 0);
        cl[CL_NC] = 0;
      }
    }
    if (!grid_barrier(bar, bar + 1, nblk, limit)) {
      if (tid == 0) post_status(status, SEEMPS_ERR_TIMEOUT);
      return;
    }
    // ---- C: apply the rotations (x' = c x - s y, y' = s x + c y, s = c t)
    const int nr = *(volatile int*)(cl + CL_NR);
    for (int k = blockIdx.x; k < nr; k += nblk) {
      const int i = cb.ri[k], j = cb.rj[k];
      const float c = cb.rc[k], s = c * cb.rt[k];
      float* xi = X + (ll)i * len;
      float* xj = X + (ll)j * len;
      for (int e = tid; e < len; e += BJ_NT) {
        const float a = xi[e], b = xj[e];
        xi[e] = fmaf(c, a, -s * b);
        xj[e] = fmaf(s, a, c * b);
      }
    }
    if (!grid_barrier(bar, bar + 1, nblk, limit)) {
      if (tid == 0) post_status(status, SEEMPS_ERR_TIMEOUT);
      return;
    }
    if (*(volatile int*)(cl + CL_ST)) break;
  }
  if (blockIdx.x == 0 && tid == 0) {
    if (rounds == CL_MAXR && cl[CL_NS] != 0) cl[CL_ST] = 1;
    cl[CL_ROUNDS] = rounds;
    const int slot = *sweeps_out;  // the block sweeps' count: this phase is recorded after them
    if (slot < max_sweeps) {
      counts[slot] = cl[CL_ROT];
      counts[max_sweeps + slot] = cl[CL_VIS];
    }
  }
}

// X[j][i] (float, column j contiguous) from the fp64 matrix M (m x n):
// columns of M (cols_of_m) or of M^T.
// Largest |M_ij| (bit pattern of a non-negative double, so an integer
// maximum is exact and order independent); *out must start at 0.
__global__ void absmax_kernel(const double* __restrict__ M, ll n, unsigned long long* out) {
  unsigned long long v = 0;
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < n; e += (ll)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(M[e]));
    v = b > v ? b : v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  if ((threadIdx.x & 31) == 0 && v) atomicMax(out, v);
}

// The scale c of the FP32 data (c = max |M_ij|, 1 for a zero matrix): the
// FP32 QR and Jacobi see M / c, so that norms and their squares stay far from
// the FP32 range limits; singular values and factors are scaled back.
__device__ __forceinline__ double noq_scale(const unsigned long long* bits) {
  const double c = __longlong_as_double((long long)*bits);
  return c > 0.0 ? c : 1.0;
}

__global__ void noq_load_kernel(const double* __restrict__ M, int m, int n, int cols_of_m,
                                const unsigned long long* __restrict__ scale, float* __restrict__ X) {
  const int len = cols_of_m ? m : n, p = cols_of_m ? n : m;
  const ll total = (ll)len * p;
  const double inv = 1.0 / noq_scale(scale);
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < total; e += (ll)gridDim.x * blockDim.x) {
    const int j = (int)(e / len), i = (int)(e % len);
    X[e] = (float)(inv * (cols_of_m ? M[(ll)i * n + j] : M[(ll)j * n + i]));
  }
}

// bf16 hi/lo split of the kept columns, scaled:  out[jj][i] = f_jj X[perm jj][i]
// with f_jj = sig_jj / s_jj^2 (the GEMM operand) ; rows padded with zeros to kp.
__global__ void noq_split_kernel(const float* __restrict__ X, int len, const int* __restrict__ perm,
                                 const double* __restrict__ sorted, const int* __restrict__ rank,
                                 const double* __restrict__ aux, int normalize, int kp, int rmax,
                                 const unsigned long long* __restrict__ scale,
                                 __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int r = *rank;
  const double c = noq_scale(scale);
  const ll total = (ll)rmax * kp;
  for (ll e = blockIdx.x * (ll)blockDim.x + threadIdx.x; e < total; e += (ll)gridDim.x * blockDim.x) {
    const int jj = (int)(e / kp), i = (int)(e % kp);
    double v = 0.0;
    if (jj < r && i < len) {
      const double s = sorted[jj];
      const double sig = normalize ? s / aux[1] : s;
      const double f = s > 0.0 ? c * sig / (s * s) : 0.0;
      v = f * (double)X[(ll)perm[jj] * len + i];
    }
    const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
  }
}

// The isometric factor from X: column jj = X[perm jj] / s_jj, written as
// rows (to_rows: out[jj][i], row stride len) or as columns (out[i][jj], row
// stride r) through a 32 x 32 shared-memory tile.
__global__ void noq_iso_kernel(const float* __restrict__ X, int len, const int* __restrict__ perm,
                               const double* __restrict__ sorted, const int* __restrict__ rank,
                               const unsigned long long* __restrict__ scale, int to_rows,
                               double* __restrict__ out) {
  __shared__ double tile[32][33];
  const int r = *rank;
  const double c = noq_scale(scale);
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  if (j0 >= r) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int jj = ty; jj < 32; jj += 8) {
    const int j = j0 + jj, i = i0 + tx;
    double v = 0.0;
    if (j < r && i < len) {
      const double s = sorted[j];
      v = s > 0.0 ? c * (double)X[(ll)perm[j] * len + i] / s : 0.0;
    }
    if (to_rows) {
      if (j < r && i < len) out[(ll)j * len + i] = v;
    } else {
      tile[jj][tx] = v;
    }
  }
  if (to_rows) return;
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + tx;
    if (i < len && j < r) out[(ll)i * r + j] = tile[tx][ii];
  }
}

// All sweeps in one CTA of 1024 threads: warp w handles pairs w, w + 32, ...
// of each step.  Used for p <= 128.
constexpr size_t SMALL_SMEM_MAX = 220 * 1024;  // dynamic shared memory of the staged small SVD
template <typename T>
__global__ void __launch_bounds__(1024) svd_small_kernel(T* __restrict__ Gg, int p, int pp,
                                                         int len, T tol, int max_sweeps,
                                                         int* __restrict__ sweeps_out, int staged) {
  __shared__ int rotated;
  extern __shared__ __align__(16) unsigned char small_smem[];
  const int lane = threadIdx.x & 31;
  const int half = threadIdx.x >> 4, hl = threadIdx.x & 15;
  const unsigned hmask = lane < 16 ? 0x0000ffffu : 0xffff0000u;
  const ll colen = (ll)len + p;
  const int colen32 = len + p;
  // staged: the whole [X; Q] array lives in shared memory for the call (the
  // rounds then wait on shared-memory rather than L2 latency)
  T* G = staged ? reinterpret_cast<T*>(small_smem) : Gg;
  if (staged) {
    for (ll e = threadIdx.x; e < colen * p; e += blockDim.x) G[e] = Gg[e];
    __syncthreads();
  }
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int step = 0; step < pp - 1; ++step) {
      // one half-warp (16 lanes) per pair: every pair of the round at once
      for (int k = half; k < pp / 2; k += 64) {
        int a, b;
        rr_pair(step, k, pp, &a, &b);
        if (a >= p || b >= p) continue;
        if (a > b) { int t = a; a = b; b = t; }
        T* xa = G + (ll)a * colen;
        T* xb = G + (ll)b * colen;
        T saa = 0, sbb = 0, sab = 0, taa = 0, tbb = 0, tab = 0;
        int i = hl;
        for (; i + 16 < len; i += 32) {
          const T u = xa[i], v = xb[i], u2 = xa[i + 16], v2 = xb[i + 16];
          saa = fma(u, u, saa);
          sbb = fma(v, v, sbb);
          sab = fma(u, v, sab);
          taa = fma(u2, u2, taa);
          tbb = fma(v2, v2, tbb);
          tab = fma(u2, v2, tab);
        }
        if (i < len) {
          const T u = xa[i], v = xb[i];
          saa = fma(u, u, saa);
          sbb = fma(v, v, sbb);
          sab = fma(u, v, sab);
        }
        saa += taa;
        sbb += tbb;
        sab += tab;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          saa += __shfl_xor_sync(hmask, saa, o);
          sbb += __shfl_xor_sync(hmask, sbb, o);
          sab += __shfl_xor_sync(hmask, sab, o);
        }
        if (sab != T(0) && fabs(sab) > tol * sqrt(saa) * sqrt(sbb)) {
          T c, s;
          jacobi_rotation<T>(saa, sbb, sab, &c, &s);
          for (int e = hl; e < colen32; e += 16) {
            const T u = xa[e], v = xb[e];
            xa[e] = c * u - s * v;
            xb[e] = s * u + c * v;
          }
          if (hl == 0) rotated = 1;
        }
        __syncwarp(hmask);
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  if (staged) {
    __syncthreads();
    for (ll e = threadIdx.x; e < colen * p; e += blockDim.x) Gg[e] = G[e];
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
// Descending order with ties broken by index: element j goes to position
// #{i : s_i > s_j or (s_i == s_j and i < j)}.  The values are non-negative, so
// their IEEE bit patterns order like the values and are compared as integers
// (FP64 compares are slow); the keys are staged in shared memory.
// (staged = false: keys read from global memory, for p above the shared budget)
constexpr int SORT_SMEM_MAX = 6144;
__global__ void svd_sort_kernel(const double* __restrict__ s, int p, int* __restrict__ perm,
                                double* __restrict__ sorted) {
  extern __shared__ long long sort_key[];
  const bool staged = p <= SORT_SMEM_MAX;
  const long long* keys = staged ? sort_key : reinterpret_cast<const long long*>(s);
  if (staged) {
    for (int i = threadIdx.x; i < p; i += blockDim.x) sort_key[i] = __double_as_longlong(s[i]);
    __syncthreads();
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x) {
    const long long v = keys[j];
    int r = 0;
    for (int i = 0; i < p; ++i) {
      const long long u = keys[i];
      r += (u > v || (u == v && i < j)) ? 1 : 0;
    }
    perm[r] = j;
    sorted[r] = s[j];
  }
}

// The truncation rule of Sect. 2.3 in a fixed summation order: the squares
// are formed in parallel, then one thread accumulates them from the
// smallest value upward (the suffix sums give the total, the tail weights
// of the scan and the discarded weight, all in that one order).
// out[0] = discarded fraction, out[1] = |S_r|; rank[0] = r.
constexpr int TR_SMEM = 4096;
__global__ void trunc_rank_kernel(const double* __restrict__ s, int n, int chi_max, double tol,
                                  int rule, int* __restrict__ rank, double* __restrict__ out) {
  __shared__ double suf[TR_SMEM];
  const bool staged = n <= TR_SMEM;
  if (staged) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) suf[j] = __dmul_rn(s[j], s[j]);
    __syncthreads();
  }
  if (threadIdx.x || blockIdx.x) return;
  int r;
  double total = 0.0;
  if (staged) {
    for (int j = n - 1; j >= 0; --j) {
      total = __dadd_rn(total, suf[j]);
      suf[j] = total;  // sum_{i >= j} s_i^2
    }
  } else {
    for (int j = n - 1; j >= 0; --j) total = __dadd_rn(total, __dmul_rn(s[j], s[j]));
  }
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
      tail = staged ? suf[j] : __dadd_rn(tail, __dmul_rn(s[j], s[j]));
      if (tail <= limit) r = j;
      else break;
    }
  }
  if (r > chi_max) r = chi_max;
  if (r < 1) r = 1;
  double kept = 0.0, disc = 0.0;
  if (staged) {
    disc = r < n ? suf[r] : 0.0;
  } else {
    for (int j = n - 1; j >= r; --j) disc = __dadd_rn(disc, __dmul_rn(s[j], s[j]));
  }
#pragma unroll 8
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
  const size_t fp64 = (len + p) * p * 8 + p * 8 * 3 + p * 4 + 4096;
  // mixed path: QR input, R^T, per-column scalars, and the GEMM's split operands
  const size_t kp = (size_t)round_up((ll)len, 64);
  const size_t mixed = 4 * (size_t)m * n + 4 * len * p + 64 * p + 4 * (p + len) * kp + 64 * 1024;
  return (fp64 > mixed ? fp64 : mixed) + 16 * 256;
}

extern "C" seemps_status seemps_truncation_rank(seemps_ctx* ctx, int n, const double* s,
                                                const seemps_strategy* st, int* rank_out) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, s && st && rank_out && n > 0, "truncation_rank: bad argument");
  SEEMPS_REQUIRE(ctx, st->chi_max >= 1, "truncation_rank: chi_max < 1");
  trunc_rank_kernel<<<1, 256, 0, ctx->stream>>>(s, n, st->chi_max, st->tol, st->rule, rank_out, nullptr);
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
      const size_t smem = ((size_t)len + p) * p * sizeof(T);
      const int staged = smem <= SMALL_SMEM_MAX ? 1 : 0;
      if (staged)  // set on every call (a cheap host call): correct for any device and thread
        SEEMPS_CHECK_CUDA(ctx, cudaFuncSetAttribute(svd_small_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)SMALL_SMEM_MAX));
      svd_small_kernel<T><<<1, 1024, staged ? smem : 0, ctx->stream>>>(G, p, pp, len, tol, max_sweeps,
                                                                       counters + max_sweeps, staged);
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
      long long limit = ctx->wait_clocks;
      void* args[] = {&G, (void*)&p, (void*)&pp, (void*)&len, &tolv, &max_sweeps, &counters, &bar,
                      &sweeps_out, &status, &limit};
      SEEMPS_CHECK_CUDA(ctx, cudaLaunchCooperativeKernel((void*)svd_coop_kernel<T>, dim3(blocks),
                                                         dim3(GT * GPB), args, 0, ctx->stream));
      SEEMPS_LAUNCHED(ctx);
    }
  }
  svd_norms_kernel<T><<<p, 256, 0, ctx->stream>>>(G, p, len, s);
  SEEMPS_LAUNCHED(ctx);
  svd_sort_kernel<<<ceil_div(p, 64), 64, p <= SORT_SMEM_MAX ? sizeof(long long) * p : 0, ctx->stream>>>(
      s, p, perm, sorted);
  SEEMPS_LAUNCHED(ctx);
  trunc_rank_kernel<<<1, 256, 0, ctx->stream>>>(sorted, p, st->chi_max, st->tol, st->rule, rank_out, aux);
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

__global__ void noq_norms_kernel(const float* __restrict__ X, int len, const unsigned long long* __restrict__ scale,
                                 double* __restrict__ s) {
  __shared__ double sh[32];
  const float* x = X + (ll)blockIdx.x * len;
  double acc = 0.0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) acc = fma((double)x[i], (double)x[i], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) s[blockIdx.x] = noq_scale(scale) * sqrt(acc);
}

template <int B, int R>
seemps_status launch_block(seemps_ctx* ctx, float* X, int p, int len, float tol, int max_sweeps,
                           int* counters, unsigned* bar, int* sweeps_out, float* nrm, int* last_mod,
                           unsigned long long* blk, int switch_rot, const CleanupBuf& cb) {
  int nb = (p + B - 1) / B;
  int nbp = nb + (nb & 1);
  int per_sm = 0;
  SEEMPS_CHECK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, svd_block_kernel<B, R>,
                                                                       BJ_NT, 0));
  int blocks = per_sm * ctx->sm_count;
  if (blocks > nbp / 2) blocks = nbp / 2;
  if (blocks < 1) {
    seemps_set_error(ctx, "svd: cooperative kernel cannot be resident");
    return SEEMPS_ERR_UNSUPPORTED;
  }
  int* status = ctx->d_status;
  long long limit = ctx->wait_clocks;
  int* cl = cb.cl;
  void* args[] = {&X, &p, &len, &nb, &nbp, &tol, &max_sweeps, &counters, &bar, &sweeps_out, &status,
                  &nrm, &last_mod, &blk, &limit, &switch_rot, &cl};
  // a power-of-two block count with a CTA per block pair: stationary blocks
  int per_sm_s = 0;
  SEEMPS_CHECK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, svd_sm_kernel<B, R>, BJ_NT, 0));
  if (nbp >= 4 && (nbp & (nbp - 1)) == 0 && nbp / 2 <= per_sm_s * ctx->sm_count) {
    SEEMPS_CHECK_CUDA(ctx, cudaLaunchCooperativeKernel((void*)svd_sm_kernel<B, R>, dim3(nbp / 2), dim3(BJ_NT), args,
                                                       0, ctx->stream));
  } else {
    SEEMPS_CHECK_CUDA(ctx, cudaLaunchCooperativeKernel((void*)svd_block_kernel<B, R>, dim3(blocks),
                                                       dim3(BJ_NT), args, 0, ctx->stream));
  }
  SEEMPS_LAUNCHED(ctx);
  if (switch_rot > 0) {
    // the cleanup phase (returns at once unless the block sweeps handed over)
    constexpr int JB = R <= 8 ? 4 : 2;
    int per_sm_c = 0;
    SEEMPS_CHECK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_c, svd_cleanup_kernel<R, JB>,
                                                                         BJ_NT, 0));
    int cblocks = (per_sm_c < 2 ? per_sm_c : 2) * ctx->sm_count;
    if (cblocks < 1) {
      seemps_set_error(ctx, "svd: cooperative cleanup kernel cannot be resident");
      return SEEMPS_ERR_UNSUPPORTED;
    }
    CleanupBuf cbuf = cb;
    const int* sw = sweeps_out;
    void* cargs[] = {&X, &p, &len, &tol, &cbuf, &last_mod, &counters, &sw, &max_sweeps, &bar, &status, &limit};
    SEEMPS_CHECK_CUDA(ctx, cudaLaunchCooperativeKernel((void*)svd_cleanup_kernel<R, JB>, dim3(cblocks),
                                                       dim3(BJ_NT), cargs, 0, ctx->stream));
    SEEMPS_LAUNCHED(ctx);
  }
  return SEEMPS_OK;
}

// bf16x3 sweep: FP32 Jacobi for the isometric side only, preconditioned by
// an FP32 QR, the other factor by one tensor-core GEMM:
//   ABSORB_RIGHT: M^T = Q R, X = R^T (m x p) -> Jacobi -> X = U S, U = X/s;
//                 A_right = diag(sig/s^2) X^T M
//   ABSORB_LEFT : M = Q R,   X = R^T (n x p) -> Jacobi -> X = V S, V = X/s;
//                 A_left = M X diag(sig/s^2)
// (p = min(m, n); sig = s or s/|S_r|).  X = R^T has the left singular
// vectors and singular values of M (resp. M^T) because M M^T = R^T R.
// Requires the isometric side length and the other dimension <= 4096.
seemps_status svd_noq_run(seemps_ctx* ctx, int m, int n, const double* theta, const seemps_strategy* st,
                          int absorb, int normalize, double* A_left, double* A_right, double* S,
                          int* rank_out, double* discarded_out, int max_sweeps) {
  const bool cols_of_m = (absorb == SEEMPS_ABSORB_RIGHT);
  // isometric side of length len; A = the matrix whose R factor is taken:
  // M^T (n x m) for ABSORB_RIGHT, M (m x n) for ABSORB_LEFT; X = R^T has
  // p = min(m, n) columns of length len
  const int len = cols_of_m ? m : n, other = cols_of_m ? n : m;
  const int p = m < n ? m : n;
  float *X, *Aq;
  double *s, *sorted, *aux;
  int *perm, *counters;
  unsigned* bar;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)len * p, &X));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)len * other, &Aq));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &s));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &sorted));
  SEEMPS_TRY(ws_alloc(ctx, 4, &aux));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &perm));
  SEEMPS_TRY(ws_alloc(ctx, 2 * (size_t)max_sweeps + 2, &counters));
  SEEMPS_TRY(ws_alloc(ctx, 4, &bar));
  const float tol = (float)fmax(Eps<float>::v * 4.0, 2.0 * sqrt((double)len) * Eps<float>::v);
  // A column-major: its columns are the rows of M (ABSORB_RIGHT) or the
  // columns of M (ABSORB_LEFT)
  unsigned long long* scale;
  SEEMPS_TRY(ws_alloc(ctx, 1, &scale));
  SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(scale, 0, sizeof(unsigned long long), ctx->stream));
  absmax_kernel<<<stride_grid(ctx, (ll)m * n, 256, 4), 256, 0, ctx->stream>>>(theta, (ll)m * n, scale);
  SEEMPS_LAUNCHED(ctx);
  noq_load_kernel<<<stride_grid(ctx, (ll)len * other, 256, 8), 256, 0, ctx->stream>>>(theta, m, n,
                                                                                      cols_of_m ? 0 : 1, scale, Aq);
  SEEMPS_LAUNCHED(ctx);
  {
    PhaseTimer qt(ctx, SEEMPS_PHASE_QR);
    SEEMPS_TRY(qr_r_transpose(ctx, Aq, other, len, X));
  }
  int* sweeps_out = counters + 2 * max_sweeps;
  // the last sweeps go to the cleanup phase once a sweep rotates at most 1/64
  // of the p (p - 1) / 2 pairs (the quadratically convergent tail; the sweep
  // after such a sweep rotates ~1/50 as many, few enough for the cleanup)
  const int switch_rot = p >= 64 ? (int)((ll)p * (p - 1) / 128) : 0;
  float* nrm = nullptr;
  int* last_mod = nullptr;
  unsigned long long* blk = nullptr;
  CleanupBuf cb = {};
  if (p > 1) {
    SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &nrm));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &last_mod));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)p + 2, &blk));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)CL_WORDS, &cb.cl));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &cb.S));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)p, &cb.mark));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)CL_CAP, &cb.ci));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)CL_CAP, &cb.cj));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)CL_CAP, &cb.cg));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)CL_CAP, &cb.ca));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)CL_CAP, &cb.cb));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)p / 2 + 1, &cb.ri));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)p / 2 + 1, &cb.rj));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)p / 2 + 1, &cb.rt));
    SEEMPS_TRY(ws_alloc(ctx, (size_t)p / 2 + 1, &cb.rc));
  }
  auto jacobi = [&](int sw) -> seemps_status {
    SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(counters, 0, sizeof(int) * (2 * max_sweeps + 2), ctx->stream));
    SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(bar, 0, sizeof(unsigned) * 4, ctx->stream));
    SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(last_mod, 0xFF, sizeof(int) * p, ctx->stream));  // -1: never rotated
    SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(blk, 0, sizeof(unsigned long long) * (p + 2), ctx->stream));
    SEEMPS_CHECK_CUDA(ctx, cudaMemsetAsync(cb.cl, 0, sizeof(int) * CL_WORDS, ctx->stream));
    PhaseTimer jt(ctx, SEEMPS_PHASE_JACOBI);
    if (len <= 2 * BJ_NT)
      return launch_block<8, 2>(ctx, X, p, len, tol, max_sweeps, counters, bar, sweeps_out, nrm, last_mod, blk, sw, cb);
    if (len <= 4 * BJ_NT)
      return launch_block<8, 4>(ctx, X, p, len, tol, max_sweeps, counters, bar, sweeps_out, nrm, last_mod, blk, sw, cb);
    if (len <= 8 * BJ_NT)
      return launch_block<8, 8>(ctx, X, p, len, tol, max_sweeps, counters, bar, sweeps_out, nrm, last_mod, blk, sw, cb);
    return launch_block<4, 16>(ctx, X, p, len, tol, max_sweeps, counters, bar, sweeps_out, nrm, last_mod, blk, sw, cb);
  };
  auto finish = [&]() -> seemps_status {
    noq_norms_kernel<<<p, 256, 0, ctx->stream>>>(X, len, scale, s);
    SEEMPS_LAUNCHED(ctx);
    svd_sort_kernel<<<ceil_div(p, 64), 64, p <= SORT_SMEM_MAX ? sizeof(long long) * p : 0, ctx->stream>>>(
        s, p, perm, sorted);
    SEEMPS_LAUNCHED(ctx);
    trunc_rank_kernel<<<1, 256, 0, ctx->stream>>>(sorted, p, st->chi_max, st->tol, st->rule, rank_out, aux);
    SEEMPS_LAUNCHED(ctx);
    if (discarded_out)
      SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(discarded_out, aux, sizeof(double), cudaMemcpyDeviceToDevice,
                                             ctx->stream));
    if (S)
      SEEMPS_CHECK_CUDA(ctx, cudaMemcpyAsync(S, sorted, sizeof(double) * p, cudaMemcpyDeviceToDevice,
                                             ctx->stream));
    return SEEMPS_OK;
  };
  if (p > 1) SEEMPS_TRY(jacobi(switch_rot));
  SEEMPS_TRY(finish());
  // the GEMM's shape depends on the rank: read it back (one sync per split)
  int r = 0;
  SEEMPS_TRY(copy_scalar_to_host(ctx, rank_out, &r, sizeof(int)));
  if (p > 1 && switch_rot > 0) {
    int clh[CL_WORDS];
    SEEMPS_TRY(copy_scalar_to_host(ctx, cb.cl, clh, sizeof(clh)));
    if (clh[CL_EN] && clh[CL_ST]) {
      // the cleanup dropped violating pairs or ran out of rounds: finish with
      // block sweeps from the current columns
      SEEMPS_TRY(jacobi(0));
      SEEMPS_TRY(finish());
      SEEMPS_TRY(copy_scalar_to_host(ctx, rank_out, &r, sizeof(int)));
      ctx->svd_cleanup_fallbacks += 1;
    } else if (clh[CL_EN]) {
      ctx->svd_cleanup_calls += 1;
      ctx->svd_cleanup_rounds += clh[CL_ROUNDS];
    }
  }
  if (p > 1) {
    // algorithmic work of the Jacobi kernel: per visited pair one dot product
    // (2 FP32 operations per element), per rotation 6 operations per element
    std::vector<int> cnt(2 * (size_t)max_sweeps + 1);
    SEEMPS_TRY(copy_scalar_to_host(ctx, counters, cnt.data(), sizeof(int) * cnt.size()));
    const int sweeps = cnt[2 * (size_t)max_sweeps];
    long long rots = 0, visits = 0;
    for (int i = 0; i < max_sweeps; ++i) {
      rots += cnt[i];
      visits += cnt[max_sweeps + i];
    }
    ctx->svd_last_n = sweeps < max_sweeps ? sweeps + 1 : sweeps;
    for (int i = 0; i < ctx->svd_last_n; ++i) {
      ctx->svd_last_rot[i] = cnt[i];
      ctx->svd_last_vis[i] = cnt[max_sweeps + i];
    }
    ctx->svd_calls += 1;
    ctx->svd_sweeps += sweeps;
    ctx->svd_pairs += visits;
    ctx->svd_flops += (double)len * (2.0 * (double)visits + 6.0 * (double)rots);
  }
  const int kp = (int)round_up(len, 64);
  __nv_bfloat16 *fh, *fl, *mh, *ml;
  SEEMPS_TRY(ws_alloc(ctx, (size_t)r * kp, &fh));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)r * kp, &fl));
  SEEMPS_TRY(ws_alloc(ctx, (size_t)other * kp, &mh));  // other = rows of the GEMM's M operand
  SEEMPS_TRY(ws_alloc(ctx, (size_t)other * kp, &ml));
  noq_split_kernel<<<stride_grid(ctx, (ll)r * kp, 256, 8), 256, 0, ctx->stream>>>(
      X, len, perm, sorted, rank_out, aux, normalize, kp, r, scale, fh, fl);
  SEEMPS_LAUNCHED(ctx);
  dim3 gi(ceil_div(len, 32), ceil_div(r, 32));
  if (cols_of_m) {
    // U (m x r) ; A_right = F M  with F = diag(f) X^T (r x m), the GEMM's B = M^T (n x m)
    noq_iso_kernel<<<gi, 256, 0, ctx->stream>>>(X, len, perm, sorted, rank_out, scale, 0, A_left);
    SEEMPS_LAUNCHED(ctx);
    SEEMPS_TRY(split_bf16(ctx, theta, n, m, n, true, mh, ml));
    SplitOperand a = {fh, fl, r};
    SplitOperand b = {mh, ml, n};
    SEEMPS_TRY(tc_gemm_f64out(ctx, a, b, kp, A_right, n));
  } else {
    // V^T (r x n) ; A_left = M F^T  with F = diag(f) X^T (r x n), the GEMM's A = M (m x n)
    noq_iso_kernel<<<gi, 256, 0, ctx->stream>>>(X, len, perm, sorted, rank_out, scale, 1, A_right);
    SEEMPS_LAUNCHED(ctx);
    SEEMPS_TRY(split_bf16(ctx, theta, n, m, n, false, mh, ml));
    SplitOperand a = {mh, ml, m};
    SplitOperand b = {fh, fl, r};
    SEEMPS_TRY(tc_gemm_f64out(ctx, a, b, kp, A_left, r));
  }
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_svd_stats(seemps_ctx* ctx, long long* calls, long long* sweeps,
                                          long long* pair_visits, double* flops, int reset) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  if (calls) *calls = ctx->svd_calls;
  if (sweeps) *sweeps = ctx->svd_sweeps;
  if (pair_visits) *pair_visits = ctx->svd_pairs;
  if (flops) *flops = ctx->svd_flops;
  if (reset) {
    ctx->svd_calls = ctx->svd_sweeps = ctx->svd_pairs = 0;
    ctx->svd_flops = 0.0;
  }
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_svd_cleanup_stats(seemps_ctx* ctx, long long* calls, long long* rounds,
                                                  long long* fallbacks, int reset) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  if (calls) *calls = ctx->svd_cleanup_calls;
  if (rounds) *rounds = ctx->svd_cleanup_rounds;
  if (fallbacks) *fallbacks = ctx->svd_cleanup_fallbacks;
  if (reset) ctx->svd_cleanup_calls = ctx->svd_cleanup_rounds = ctx->svd_cleanup_fallbacks = 0;
  return SEEMPS_OK;
}

extern "C" seemps_status seemps_svd_sweep_counts(seemps_ctx* ctx, int* rotations, int* visits, int cap,
                                                 int* n_sweeps) {
  if (!ctx) return SEEMPS_ERR_INVALID;
  SEEMPS_REQUIRE(ctx, cap >= 0, "svd_sweep_counts: negative capacity");
  const int n = ctx->svd_last_n;
  for (int i = 0; i < n && i < cap; ++i) {
    if (rotations) rotations[i] = ctx->svd_last_rot[i];
    if (visits) visits[i] = ctx->svd_last_vis[i];
  }
  if (n_sweeps) *n_sweeps = n;
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
  SEEMPS_REQUIRE(ctx, precision == SEEMPS_FP64 || precision == SEEMPS_BF16X3 || precision == SEEMPS_FP64X2,
                 "svd_truncate: unknown precision");
  if (max_sweeps <= 0) max_sweeps = 40;
  if (max_sweeps > SEEMPS_MAX_JACOBI_SWEEPS) max_sweeps = SEEMPS_MAX_JACOBI_SWEEPS;
  WsFrame frame(ctx);
  PhaseTimer timer(ctx, SEEMPS_PHASE_SVD);
  if (precision != SEEMPS_BF16X3)  // FP64X2 splits in FP64 (its double-FP64 part is the environments)
    return svd_run<double>(ctx, m, n, theta, st, absorb, normalize, A_left, A_right, S, rank_out,
                           discarded_out, max_sweeps);
  // bf16x3 sweep: Jacobi on the isometric side only when that side is the
  // narrower one (large problems); otherwise the accumulated-rotation path
  const int iso_other = (absorb == SEEMPS_ABSORB_RIGHT) ? n : m;
  const int iso_len = (absorb == SEEMPS_ABSORB_RIGHT) ? m : n;
  const int kmin = m < n ? m : n;
  if (kmin > 128 && iso_len <= 4096 && qr_supported(iso_other, iso_len) && tc_available(ctx))
    return svd_noq_run(ctx, m, n, theta, st, absorb, normalize, A_left, A_right, S, rank_out,
                       discarded_out, max_sweeps);
  return svd_run<float>(ctx, m, n, theta, st, absorb, normalize, A_left, A_right, S, rank_out,
                        discarded_out, max_sweeps);
}
