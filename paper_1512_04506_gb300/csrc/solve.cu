// Coarse-grid solve of Alg. 2: restarted FGMRES(m) on D_c with classical Gram-Schmidt Arnoldi
// and Givens rotations, one independent Krylov space per right-hand side.  Vectors stay in the
// coarse layout [Vc][2][ntv][nrhs]; all scalars (Hessenberg matrix, rotations, residual
// estimates, convergence flags) live on the device, so the host only launches kernels.
//
// One Arnoldi step is two launches for nrhs in {1, 2, 4, 8, 16}: w = D_c V_j (the application
// reads the unnormalised vector times 1/h_{j,j-1} and stores V_j on the way), then the
// cooperative k_arnoldi (dots <V_i, w>, column j of H, w -= sum H_ij V_i with |w|^2, Givens
// rotation and convergence test, phases separated by grid barriers).  Other column counts take
// three launches (k_dots, then k_update, each ending in a last-CTA reduction).  Once every
// right-hand side has converged the device flag `done` makes every later kernel return at once
// and a mapped host word receives the solve's ticket; the host reads it after the next
// application is queued (so the GPU never waits for the host) or, without polling, launches the
// whole budget.
#include "amg_internal.cuh"

#include <algorithm>

namespace {

constexpr int ST_T = 256;
constexpr int MAXR = 16;
constexpr int kMaxPartRows = 1024;  // most CTAs of the partial-sum kernels (rows of FState::part)

// CTAs of the partial-sum kernels (k_dots, k_update, k_residual): two per SM.
int solve_nblk() { return std::min(2 * amg_sm_count(), kMaxPartRows); }

struct FState {
  int m, nrhs, nblk;
  long long rows;  // Vc * nc
  double tol;
  double2 *H, *cs, *sn, *gv, *part;
  double *bnorm, *relres, *invh;
  int *active, *kcnt, *applies, *done;
  unsigned* counter;
  unsigned* bar;     // grid barrier of k_arnoldi: [0] arrivals, [1] generation
  unsigned* err;     // device error word
  volatile int* hdone;  // mapped host word: set to `ticket` when every right-hand side has converged
  int ticket;
  unsigned bar_extra;  // 0, or the test hook's arrivals that never come
};

// Every right-hand side has converged: later kernels of this solve return at once, and the host
// (which polls the mapped word after an event) stops launching.
__device__ inline void mark_done(FState& s) {
  *s.done = 1;
  if (s.hdone) *s.hdone = s.ticket;
}

__device__ inline double2 to_d(float2 v) { return make_double2(v.x, v.y); }
__device__ inline double2 to_d(double2 v) { return v; }
template <typename CT> __device__ inline CT from_d(double2 v);
template <> __device__ inline float2 from_d<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ inline double2 from_d<double2>(double2 v) { return v; }

__device__ inline double2 ld_cg(const double2* p) { return __ldcg(p); }

// CTA-wide sum of nrhs complex values per thread; thread r < nrhs writes out[r].
__device__ inline void cta_sum_store(double2 (&acc)[MAXR], int nrhs, double2* out) {
  __shared__ double2 sm[ST_T / 32][MAXR];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < MAXR; ++r) {
    if (r >= nrhs) break;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, o);
      acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, o);
    }
    if (lane == 0) sm[warp][r] = acc[r];
  }
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double2 t = make_double2(0, 0);
    for (int w = 0; w < ST_T / 32; ++w) t = cadd(t, sm[w][threadIdx.x]);
    out[threadIdx.x] = t;
  }
}

// Last-CTA election: every CTA publishes its partial sums, then counts itself in; the CTA that
// brings the count to `total` sees every partial (threadfence before the count) and resets it.
__device__ inline bool last_block(unsigned* counter, unsigned total) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(counter, 1u);
    last = prev == total - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) *counter = 0;
  return last;
}

// Sum over the nblk partials of pair t (layout part[(i * nblk + b) * nrhs + r], t = i * nrhs + r)
// by one warp: lanes stride over the partials, then a shuffle sum; valid in lane 0.
__device__ inline double2 warp_sum_partials(const double2* part, int nblk, int nrhs, int t) {
  const int lane = threadIdx.x & 31;
  const int i = t / nrhs, r = t % nrhs;
  double2 sum = make_double2(0, 0);
  for (int b = lane; b < nblk; b += 32) sum = cadd(sum, ld_cg(part + ((long long)i * nblk + b) * nrhs + r));
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    sum.x += __shfl_xor_sync(0xffffffffu, sum.x, o);
    sum.y += __shfl_xor_sync(0xffffffffu, sum.y, o);
  }
  return sum;
}

// ---- flat forms for nrhs dividing 32 (2, 4, 8, 16): the loops run over e = row * nrhs + r with
// consecutive threads on consecutive elements (coalesced), and since the stride and every warp's
// first element are multiples of 32, a thread only ever meets column e % nrhs = lane % nrhs.
// Per-column sums: xor shuffles over the lanes of equal column, then over the warps.
__device__ inline void cta_col_sum_store(double2 v, int nrhs, double2* out) {
  __shared__ double2 sm[ST_T / 32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o >= nrhs; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  if (lane < nrhs) sm[warp][lane] = v;
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double2 t = make_double2(0, 0);
    for (int w = 0; w < ST_T / 32; ++w) t = cadd(t, sm[w][threadIdx.x]);
    out[threadIdx.x] = t;
  }
}

__device__ inline double2 shfl_d2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Givens rotation and convergence test of Arnoldi step j for right-hand side r, given |w|^2 = n2,
// by one warp (restart length <= 64): lane l fetches entries l and l + 32 of the new Hessenberg
// column and of the earlier rotations in one round of loads.  Applying the earlier rotations to
// the column is a linear recurrence in the entry carried from rotation i to i + 1:
// carry_{i+1} = conj(c_i) col[i+1] - conj(s_i) carry_i, carry_0 = col[0], and the finished
// entries are c_i carry_i + s_i col[i+1].  The carries are a prefix composition of the complex
// affine maps x -> A_i + B_i x, taken as a warp scan (five shuffle rounds per 32 rotations)
// instead of a chain of j dependent steps.
__device__ inline void givens_scan_half(const double2& ci, const double2& si, const double2& b, bool valid, double2 x0,
                                        double2& carry_i, double2& carry_next) {
  const int lane = threadIdx.x & 31;
  double2 A = valid ? cmulc(ci, b) : make_double2(0, 0);               // conj(c_i) b
  double2 Bm = valid ? make_double2(-si.x, si.y) : make_double2(1, 0);  // -conj(s_i)
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double2 Ap = make_double2(__shfl_up_sync(0xffffffffu, A.x, o), __shfl_up_sync(0xffffffffu, A.y, o));
    const double2 Bp = make_double2(__shfl_up_sync(0xffffffffu, Bm.x, o), __shfl_up_sync(0xffffffffu, Bm.y, o));
    if (lane >= o) {
      A = cadd(A, cmul(Bm, Ap));
      Bm = cmul(Bm, Bp);
    }
  }
  carry_next = cadd(A, cmul(Bm, x0));
  const double2 prev = make_double2(__shfl_up_sync(0xffffffffu, carry_next.x, 1),
                                    __shfl_up_sync(0xffffffffu, carry_next.y, 1));
  carry_i = lane == 0 ? x0 : prev;
}

__device__ void arnoldi_step_warp(FState& s, int r, int j, double n2, int* any) {
  const int lane = threadIdx.x & 31;
  const double2 z = make_double2(0, 0);
  double2* Hc = s.H + (long long)r * (s.m + 1) * s.m;
  double2* cs = s.cs + (long long)r * s.m;
  double2* sn = s.sn + (long long)r * s.m;
  double2* gv = s.gv + (long long)r * (s.m + 1);
  const int act = __ldcg(s.active + r);
  const double rel_j = __ldcg(s.relres + r);  // |g_j| / |b|
  const int napp = __ldcg(s.applies + r);
  const double2 gj = ld_cg(gv + j);
  const double2 col0 = lane <= j ? ld_cg(Hc + lane * s.m + j) : z;
  const double2 col1 = lane + 32 <= j ? ld_cg(Hc + (lane + 32) * s.m + j) : z;
  const double2 c0 = lane < j ? ld_cg(cs + lane) : z, s0 = lane < j ? ld_cg(sn + lane) : z;
  const double2 c1 = lane + 32 < j ? ld_cg(cs + lane + 32) : z, s1 = lane + 32 < j ? ld_cg(sn + lane + 32) : z;
  if (!act) {
    if (lane == 0) s.invh[r] = 0;
    return;
  }
  const double hnext = sqrt(n2);
  // col[i + 1] for rotation i = lane (first half) and i = lane + 32 (second half)
  const double2 c32 = shfl_d2(col1, 0);
  double2 b0 = make_double2(__shfl_down_sync(0xffffffffu, col0.x, 1), __shfl_down_sync(0xffffffffu, col0.y, 1));
  if (lane == 31) b0 = c32;
  const double2 b1 = make_double2(__shfl_down_sync(0xffffffffu, col1.x, 1), __shfl_down_sync(0xffffffffu, col1.y, 1));
  const double2 x0 = shfl_d2(col0, 0);
  double2 ci0, cn0, carry = x0, f0 = z, f1 = z;
  givens_scan_half(c0, s0, b0, lane < j, x0, ci0, cn0);
  if (lane < j) f0 = cadd(cmul(c0, ci0), cmul(s0, b0));
  if (j > 0 && j <= 32) carry = shfl_d2(cn0, j - 1);
  if (j > 32) {
    const double2 x32 = shfl_d2(cn0, 31);
    double2 ci1, cn1;
    givens_scan_half(c1, s1, b1, lane + 32 < j, x32, ci1, cn1);
    if (lane + 32 < j) f1 = cadd(cmul(c1, ci1), cmul(s1, b1));
    carry = shfl_d2(cn1, j - 33);
  }
  const double den2 = carry.x * carry.x + carry.y * carry.y + n2;
  const double inv_den = den2 > 0 ? 1.0 / sqrt(den2) : 0.0;
  const double den = den2 * inv_den;
  const double2 c = den2 > 0 ? cscale(cconj(carry), inv_den) : make_double2(1, 0);
  const double2 sv = make_double2(hnext * inv_den, 0);
  if (lane < j) Hc[lane * s.m + j] = f0;
  if (lane + 32 < j) Hc[(lane + 32) * s.m + j] = f1;
  if (lane == 0) {
    Hc[j * s.m + j] = make_double2(den, 0);
    Hc[(j + 1) * s.m + j] = z;
    cs[j] = c;
    sn[j] = sv;
    const double2 g1 = cscale(cmul(cconj(sv), gj), -1.0);
    gv[j + 1] = g1;
    gv[j] = cmul(c, gj);
    const double rel = rel_j * sv.x;  // |g_{j+1}| = |s_j| |g_j|
    s.relres[r] = rel;
    s.kcnt[r] = j + 1;
    s.applies[r] = napp + 1;
    if (rel <= s.tol || hnext == 0) {
      s.active[r] = 0;
      s.invh[r] = 0;
    } else {
      s.invh[r] = 1.0 / hnext;
      atomicOr(any, 1);
    }
  }
}

// part[(i * nblk + b) * nrhs + r] = partial <V_i, w> (i = blockIdx.y); the last CTA writes H[.][i][j].
template <typename CT>
__global__ void __launch_bounds__(ST_T) k_dots(FState s, const CT* __restrict__ w, const CT* __restrict__ V,
                                               long long vstride, int j) {
  if (*s.done) return;
  const int i = blockIdx.y;
  const CT* Vi = V + i * vstride;
  CT a[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) a[r] = CT{0, 0};
  for (long long row = blockIdx.x * (long long)ST_T + threadIdx.x; row < s.rows;
       row += (long long)s.nblk * ST_T) {
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      if (r >= s.nrhs) break;
      cfmac(a[r], Vi[row * s.nrhs + r], w[row * s.nrhs + r]);
    }
  }
  double2 acc[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) acc[r] = to_d(a[r]);
  cta_sum_store(acc, s.nrhs, s.part + ((long long)i * s.nblk + blockIdx.x) * s.nrhs);
  if (!last_block(s.counter, s.nblk * (j + 1))) return;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = warp; t < (j + 1) * s.nrhs; t += nw) {
    const double2 sum = warp_sum_partials(s.part, s.nblk, s.nrhs, t);
    const int ii = t / s.nrhs, r = t % s.nrhs;
    if ((threadIdx.x & 31) == 0) s.H[((long long)r * (s.m + 1) + ii) * s.m + j] = s.active[r] ? sum : make_double2(0, 0);
  }
}

// w -= sum_{i<=j} H[r][i][j] V_i and |w|^2; the last CTA does the Givens step (arnoldi_step_warp).
template <typename CT>
__global__ void __launch_bounds__(ST_T) k_update(FState s, CT* __restrict__ w, const CT* __restrict__ V,
                                                 long long vstride, int j) {
  if (*s.done) return;
  __shared__ CT hc[AMG_MAX_NTV + 1][MAXR];
  for (int e = threadIdx.x; e < (j + 1) * s.nrhs; e += ST_T) {
    const int i = e / s.nrhs, r = e % s.nrhs;
    hc[i][r] = from_d<CT>(ld_cg(s.H + ((long long)r * (s.m + 1) + i) * s.m + j));
  }
  __syncthreads();
  CT a[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) a[r] = CT{0, 0};
  for (long long row = blockIdx.x * (long long)ST_T + threadIdx.x; row < s.rows;
       row += (long long)s.nblk * ST_T) {
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      if (r >= s.nrhs) break;
      CT v = w[row * s.nrhs + r];
      for (int i = 0; i <= j; ++i) {
        const CT q = V[i * vstride + row * s.nrhs + r];
        const CT c = hc[i][r];
        v.x -= c.x * q.x - c.y * q.y;
        v.y -= c.x * q.y + c.y * q.x;
      }
      w[row * s.nrhs + r] = v;
      a[r].x += v.x * v.x + v.y * v.y;
    }
  }
  double2 acc[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) acc[r] = to_d(a[r]);
  cta_sum_store(acc, s.nrhs, s.part + (long long)blockIdx.x * s.nrhs);
  if (!last_block(s.counter, s.nblk)) return;
  __shared__ int any;
  __shared__ double n2s[MAXR];
  if (threadIdx.x == 0) any = 0;
  for (int r = threadIdx.x >> 5; r < s.nrhs; r += blockDim.x >> 5) {
    const double2 v = warp_sum_partials(s.part, s.nblk, s.nrhs, r);
    if ((threadIdx.x & 31) == 0) n2s[r] = v.x;
  }
  __syncthreads();
  for (int r = threadIdx.x >> 5; r < s.nrhs; r += ST_T / 32) arnoldi_step_warp(s, r, j, n2s[r], &any);
  __syncthreads();
  if (threadIdx.x == 0 && !any) mark_done(s);
}

template <typename CT>
__global__ void __launch_bounds__(ST_T) k_dots_flat(FState s, const CT* __restrict__ w, const CT* __restrict__ V,
                                                    long long vstride, int j) {
  if (*s.done) return;
  const int i = blockIdx.y;
  const CT* Vi = V + i * vstride;
  const long long n = s.rows * s.nrhs;
  CT a = CT{0, 0};
  for (long long e = blockIdx.x * (long long)ST_T + threadIdx.x; e < n; e += (long long)s.nblk * ST_T)
    cfmac(a, Vi[e], w[e]);
  cta_col_sum_store(to_d(a), s.nrhs, s.part + ((long long)i * s.nblk + blockIdx.x) * s.nrhs);
  if (!last_block(s.counter, s.nblk * (j + 1))) return;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = warp; t < (j + 1) * s.nrhs; t += nw) {
    const double2 sum = warp_sum_partials(s.part, s.nblk, s.nrhs, t);
    const int ii = t / s.nrhs, r = t % s.nrhs;
    if ((threadIdx.x & 31) == 0) s.H[((long long)r * (s.m + 1) + ii) * s.m + j] = s.active[r] ? sum : make_double2(0, 0);
  }
}

template <typename CT>
__global__ void __launch_bounds__(ST_T) k_update_flat(FState s, CT* __restrict__ w, const CT* __restrict__ V,
                                                      long long vstride, int j) {
  if (*s.done) return;
  __shared__ CT hc[AMG_MAX_NTV + 1][MAXR];
  for (int e = threadIdx.x; e < (j + 1) * s.nrhs; e += ST_T) {
    const int i = e / s.nrhs, r = e % s.nrhs;
    hc[i][r] = from_d<CT>(ld_cg(s.H + ((long long)r * (s.m + 1) + i) * s.m + j));
  }
  __syncthreads();
  const int col = threadIdx.x % s.nrhs;
  const long long n = s.rows * s.nrhs;
  decltype(CT{}.x) acc = 0;
  for (long long e = blockIdx.x * (long long)ST_T + threadIdx.x; e < n; e += (long long)s.nblk * ST_T) {
    CT v = w[e];
    for (int i = 0; i <= j; ++i) {
      const CT q = V[i * vstride + e];
      const CT c = hc[i][col];
      v.x -= c.x * q.x - c.y * q.y;
      v.y -= c.x * q.y + c.y * q.x;
    }
    w[e] = v;
    acc += v.x * v.x + v.y * v.y;
  }
  cta_col_sum_store(make_double2((double)acc, 0.0), s.nrhs, s.part + (long long)blockIdx.x * s.nrhs);
  if (!last_block(s.counter, s.nblk)) return;
  __shared__ int any;
  __shared__ double n2s[MAXR];
  if (threadIdx.x == 0) any = 0;
  for (int r = threadIdx.x >> 5; r < s.nrhs; r += blockDim.x >> 5) {
    const double2 v = warp_sum_partials(s.part, s.nblk, s.nrhs, r);
    if ((threadIdx.x & 31) == 0) n2s[r] = v.x;
  }
  __syncthreads();
  for (int r = threadIdx.x >> 5; r < s.nrhs; r += ST_T / 32) arnoldi_step_warp(s, r, j, n2s[r], &any);
  __syncthreads();
  if (threadIdx.x == 0 && !any) mark_done(s);
}

// ---- fused Arnoldi step for nrhs in {1, 2, 4, 8, 16} (flat element loops as above): one
// cooperative launch, one CTA per SM, does the dots, the Hessenberg column, the update with |w|^2
// and the Givens step, with two grid barriers in place of a kernel boundary and a last-CTA
// hand-off.  With one or a few columns the coarse vectors are small (Vc * 2 Ntv rows, about a
// megabyte), each phase is a few memory round trips and the launch and barrier latencies set the
// time; with 16 columns they reach hundreds of megabytes and the phases stream, which is what the
// round shapes below are for.
constexpr int AR_T = 512;
constexpr int AR_W = AR_T / 32;
template <typename CT>
constexpr int ar_ic() { return sizeof(CT) == 8 ? 8 : 4; }  // dot products reduced per CTA round
// Round shapes of k_arnoldi: IC basis vectors per dot-product round, U elements per thread whose
// loads are issued together, KQ basis vectors per update round.  Vectors of more than
// AR_LONG elements (16 columns at 32^3 x 64 and up) take fewer basis vectors and more elements
// per round, for more loads in flight per thread at the same register count.
constexpr long long AR_LONG = 1LL << 20;
template <typename CT>
constexpr int ar_ulong() { return sizeof(CT) == 8 ? 16 : 8; }
constexpr long long kBarCycles = 2000000000LL;  // about one second at GB300 clocks

// Bounded grid barrier (every CTA resident: cooperative launch).  Thread 0 reads the generation
// before it arrives; the last arrival resets the count and advances the generation.  A wait that
// runs out sets AMG_EBIT_TIMEOUT and returns false.  `extra` > 0 (a test hook) expects arrivals
// that never come, so that every wait runs out.
__device__ bool grid_sync(unsigned* bar, unsigned* err, unsigned extra) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    int good = 1;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1 + extra) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > kBarCycles) {
          atomicOr(err, AMG_EBIT_TIMEOUT);
          good = 0;
          break;
        }
      }
      __threadfence();
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <typename CT, int AR_IC, int AR_U, int KQ>
__global__ void __launch_bounds__(AR_T) k_arnoldi(FState s, CT* __restrict__ w, const CT* __restrict__ V,
                                                  long long vstride, int j) {
  using RT = decltype(CT{}.x);
  if (*s.done) return;
  __shared__ double2 red[AR_IC][AR_W][MAXR];
  __shared__ CT hc[AMG_MAX_NTV + 1][MAXR];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nr = s.nrhs, G = gridDim.x;
  const long long n = s.rows * nr;
  const long long e0 = (long long)blockIdx.x * AR_T + threadIdx.x, es = (long long)G * AR_T;
  // 1. per-CTA partial sums of <V_i, w>, i = 0..j (lane l only ever meets column l % nr)
  for (int i0 = 0; i0 <= j; i0 += AR_IC) {
    const int ni = min(AR_IC, j + 1 - i0);
    CT a[AR_IC];
#pragma unroll
    for (int ii = 0; ii < AR_IC; ++ii) a[ii] = CT{0, 0};
    for (long long eb = e0; eb < n; eb += AR_U * es) {
      // every load of the round first (predicated), then the arithmetic
      CT wv[AR_U], vv[AR_IC][AR_U];
#pragma unroll
      for (int u = 0; u < AR_U; ++u) wv[u] = eb + u * es < n ? w[eb + u * es] : CT{0, 0};
#pragma unroll
      for (int ii = 0; ii < AR_IC; ++ii)
#pragma unroll
        for (int u = 0; u < AR_U; ++u)
          vv[ii][u] = (ii < ni && eb + u * es < n) ? V[(i0 + ii) * vstride + eb + u * es] : CT{0, 0};
#pragma unroll
      for (int ii = 0; ii < AR_IC; ++ii)
#pragma unroll
        for (int u = 0; u < AR_U; ++u) cfmac(a[ii], vv[ii][u], wv[u]);
    }
    // warp sums in the vectors' own precision (FP64 arithmetic is scarce on this GPU), then FP64
#pragma unroll
    for (int ii = 0; ii < AR_IC; ++ii) {
      if (ii < ni) {
        CT v = a[ii];
        for (int o = 16; o >= nr; o >>= 1) {
          v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
          v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        }
        if (lane < nr) red[ii][warp][lane] = to_d(v);
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ni * nr; t += AR_T) {
      const int ii = t / nr, r = t % nr;
      double2 sum = make_double2(0, 0);
      for (int wp = 0; wp < AR_W; ++wp) sum = cadd(sum, red[ii][wp][r]);
      s.part[((long long)(i0 + ii) * G + blockIdx.x) * nr + r] = sum;
    }
    __syncthreads();
  }
  if (!grid_sync(s.bar, s.err, s.bar_extra)) return;
  // 2. column j of H: one warp per (i, r) sums the G partials
  const int P = (j + 1) * nr;
  for (int t = blockIdx.x * AR_W + warp; t < P; t += G * AR_W) {
    const double2 sum = warp_sum_partials(s.part, G, nr, t);
    const int i = t / nr, r = t % nr;
    if (lane == 0) s.H[((long long)r * (s.m + 1) + i) * s.m + j] = __ldcg(s.active + r) ? sum : make_double2(0, 0);
  }
  if (!grid_sync(s.bar, s.err, s.bar_extra)) return;
  // 3. w -= sum_i H[r][i][j] V_i and the partial sums of |w|^2 (into row 0 of the partials,
  // whose reads in 2. are complete)
  for (int t = threadIdx.x; t < P; t += AR_T) {
    const int i = t / nr, r = t % nr;
    hc[i][r] = from_d<CT>(ld_cg(s.H + ((long long)r * (s.m + 1) + i) * s.m + j));
  }
  __syncthreads();
  const int col = lane % nr;
  RT acc = 0;
  for (long long eb = e0; eb < n; eb += AR_U * es) {
    CT v[AR_U];
#pragma unroll
    for (int u = 0; u < AR_U; ++u) v[u] = eb + u * es < n ? w[eb + u * es] : CT{0, 0};
    // KQ basis vectors per round of loads
    int i = 0;
    for (; i + KQ <= j + 1; i += KQ) {
      CT q[KQ][AR_U];
#pragma unroll
      for (int k = 0; k < KQ; ++k)
#pragma unroll
        for (int u = 0; u < AR_U; ++u) q[k][u] = eb + u * es < n ? V[(i + k) * vstride + eb + u * es] : CT{0, 0};
#pragma unroll
      for (int k = 0; k < KQ; ++k) {
        const CT c = hc[i + k][col];
#pragma unroll
        for (int u = 0; u < AR_U; ++u) {
          v[u].x -= c.x * q[k][u].x - c.y * q[k][u].y;
          v[u].y -= c.x * q[k][u].y + c.y * q[k][u].x;
        }
      }
    }
    for (; i <= j; ++i) {
      const CT c = hc[i][col];
      CT q[AR_U];
#pragma unroll
      for (int u = 0; u < AR_U; ++u) q[u] = eb + u * es < n ? V[i * vstride + eb + u * es] : CT{0, 0};
#pragma unroll
      for (int u = 0; u < AR_U; ++u) {
        v[u].x -= c.x * q[u].x - c.y * q[u].y;
        v[u].y -= c.x * q[u].y + c.y * q[u].x;
      }
    }
#pragma unroll
    for (int u = 0; u < AR_U; ++u)
      if (eb + u * es < n) {
        w[eb + u * es] = v[u];
        acc += v[u].x * v[u].x + v[u].y * v[u].y;
      }
  }
  for (int o = 16; o >= nr; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane < nr) red[0][warp][lane] = make_double2((double)acc, 0);
  __syncthreads();
  if (threadIdx.x < nr) {
    double sum = 0;
    for (int wp = 0; wp < AR_W; ++wp) sum += red[0][wp][threadIdx.x].x;
    s.part[(long long)blockIdx.x * nr + threadIdx.x] = make_double2(sum, 0);
  }
  // 4. the last CTA: |w|^2 per column and the Givens step, one warp per right-hand side
  if (!last_block(s.counter, G)) return;
  __shared__ int any;
  __shared__ double n2s[MAXR];
  if (threadIdx.x == 0) any = 0;
  for (int r = warp; r < nr; r += AR_W) {
    const double2 v = warp_sum_partials(s.part, G, nr, r);
    if (lane == 0) n2s[r] = v.x;
  }
  __syncthreads();
  for (int r = warp; r < nr; r += AR_W) arnoldi_step_warp(s, r, j, n2s[r], &any);
  __syncthreads();
  if (threadIdx.x == 0 && !any) mark_done(s);
}

// End of a cycle: every CTA solves the small triangular systems R y = g (one warp per right-hand
// side, column by column from the last: lane l holds the residual entries l and l + 32 of g, and
// the next column's loads are issued before the current one is used), then x += sum_i y_i V_i
// over the columns built in the cycle.  The last CTA resets the column counts, so a repeated call
// adds nothing (after convergence the restart residual returns at once and does not reset them).
template <typename CT>
__global__ void __launch_bounds__(ST_T) k_xupdate(FState s, CT* __restrict__ x, const CT* __restrict__ V,
                                                  long long vstride) {
  __shared__ double2 yd[MAXR][AMG_MAX_NTV];
  __shared__ CT yc[AMG_MAX_NTV][MAXR];
  __shared__ int kmax;
  const int lane = threadIdx.x & 31;
  const double2 z = make_double2(0, 0);
  if (threadIdx.x == 0) kmax = 0;
  __syncthreads();
  for (int r = threadIdx.x >> 5; r < s.nrhs; r += ST_T / 32) {
    const int k = __ldcg(s.kcnt + r);
    const double2* Hc = s.H + (long long)r * (s.m + 1) * s.m;
    const double2* gv = s.gv + (long long)r * (s.m + 1);
    double2 t0 = lane < k ? ld_cg(gv + lane) : z, t1 = lane + 32 < k ? ld_cg(gv + lane + 32) : z;
    for (int i = k + lane; i < s.m; i += 32) yd[r][i] = z;
    int i = k - 1;
    double2 h0 = z, h1 = z, dg = z;
    if (i >= 0) {
      h0 = lane < i ? ld_cg(Hc + lane * s.m + i) : z;
      h1 = lane + 32 < i ? ld_cg(Hc + (lane + 32) * s.m + i) : z;
      dg = ld_cg(Hc + i * s.m + i);
    }
    for (; i >= 0; --i) {
      double2 n0 = z, n1 = z, nd = z;
      if (i > 0) {
        n0 = lane < i - 1 ? ld_cg(Hc + lane * s.m + i - 1) : z;
        n1 = lane + 32 < i - 1 ? ld_cg(Hc + (lane + 32) * s.m + i - 1) : z;
        nd = ld_cg(Hc + (i - 1) * s.m + i - 1);
      }
      const double2 ti = shfl_d2(i < 32 ? t0 : t1, i & 31);
      const double dd = dg.x * dg.x + dg.y * dg.y;
      const double2 yi = dd > 0 ? cscale(cmulc(dg, ti), 1.0 / dd) : z;
      if (lane == 0) yd[r][i] = yi;
      if (lane < i) t0 = csub(t0, cmul(h0, yi));
      if (lane + 32 < i) t1 = csub(t1, cmul(h1, yi));
      h0 = n0;
      h1 = n1;
      dg = nd;
    }
    if (lane == 0) atomicMax(&kmax, k);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < s.m * s.nrhs; e += blockDim.x) {
    const int i = e / s.nrhs, r = e % s.nrhs;
    yc[i][r] = from_d<CT>(yd[r][i]);
  }
  __syncthreads();
  const int km = kmax;
  const long long n = s.rows * s.nrhs;
  if (km > 0) {
    // four elements per thread and four basis vectors per round of loads
    const long long es = (long long)gridDim.x * blockDim.x;
    for (long long eb = blockIdx.x * (long long)blockDim.x + threadIdx.x; eb < n; eb += 4 * es) {
      CT v[4];
      int rr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        v[u] = eb + u * es < n ? x[eb + u * es] : CT{0, 0};
        rr[u] = (int)((eb + u * es) % s.nrhs);
      }
      int i = 0;
      for (; i + 4 <= km; i += 4) {
        CT q[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int u = 0; u < 4; ++u) q[k][u] = eb + u * es < n ? V[(i + k) * vstride + eb + u * es] : CT{0, 0};
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const CT c = yc[i + k][rr[u]];
            v[u].x += c.x * q[k][u].x - c.y * q[k][u].y;
            v[u].y += c.x * q[k][u].y + c.y * q[k][u].x;
          }
      }
      for (; i < km; ++i) {
        CT q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = eb + u * es < n ? V[i * vstride + eb + u * es] : CT{0, 0};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const CT c = yc[i][rr[u]];
          v[u].x += c.x * q[u].x - c.y * q[u].y;
          v[u].y += c.x * q[u].y + c.y * q[u].x;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (eb + u * es < n) x[eb + u * es] = v[u];
    }
  }
  if (!last_block(s.counter, gridDim.x)) return;
  if (threadIdx.x < s.nrhs) s.kcnt[threadIdx.x] = 0;
}

// w = b - w (restart residual; first = 1: w = b) and |w|^2; the last CTA starts the cycle:
// beta = |r|, convergence test, g = (beta, 0, ...), invh = 1 / beta.
template <typename CT>
__global__ void __launch_bounds__(ST_T) k_residual(FState s, CT* __restrict__ w, const CT* __restrict__ b, int first,
                                                   CT* __restrict__ xzero) {
  if (*s.done) return;
  if (32 % s.nrhs == 0) {  // flat, coalesced (see k_dots_flat; one column included)
    const long long n = s.rows * s.nrhs, es = (long long)s.nblk * ST_T;
    decltype(CT{}.x) acc = 0;
    for (long long eb = blockIdx.x * (long long)ST_T + threadIdx.x; eb < n; eb += 4 * es) {  // 4 elements per round
      CT v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long e = eb + u * es;
        v[u] = e < n ? b[e] : CT{0, 0};
        if (!first && e < n) {
          const CT q = w[e];
          v[u].x -= q.x;
          v[u].y -= q.y;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long e = eb + u * es;
        if (e < n) {
          w[e] = v[u];
          if (xzero) xzero[e] = CT{0, 0};
          acc += v[u].x * v[u].x + v[u].y * v[u].y;
        }
      }
    }
    cta_col_sum_store(make_double2((double)acc, 0.0), s.nrhs, s.part + (long long)blockIdx.x * s.nrhs);
  } else {
    CT a[MAXR];
#pragma unroll
    for (int r = 0; r < MAXR; ++r) a[r] = CT{0, 0};
    for (long long row = blockIdx.x * (long long)ST_T + threadIdx.x; row < s.rows;
         row += (long long)s.nblk * ST_T) {
#pragma unroll
      for (int r = 0; r < MAXR; ++r) {
        if (r >= s.nrhs) break;
        CT v = b[row * s.nrhs + r];
        if (!first) {
          const CT q = w[row * s.nrhs + r];
          v.x -= q.x;
          v.y -= q.y;
        }
        w[row * s.nrhs + r] = v;
        if (xzero) xzero[row * s.nrhs + r] = CT{0, 0};
        a[r].x += v.x * v.x + v.y * v.y;
      }
    }
    double2 acc[MAXR];
#pragma unroll
    for (int r = 0; r < MAXR; ++r) acc[r] = to_d(a[r]);
    cta_sum_store(acc, s.nrhs, s.part + (long long)blockIdx.x * s.nrhs);
  }
  if (!last_block(s.counter, s.nblk)) return;
  __shared__ int any;
  __shared__ double n2s[MAXR];
  if (threadIdx.x == 0) any = 0;
  for (int r = threadIdx.x >> 5; r < s.nrhs; r += blockDim.x >> 5) {
    const double2 v = warp_sum_partials(s.part, s.nblk, s.nrhs, r);
    if ((threadIdx.x & 31) == 0) n2s[r] = v.x;
  }
  __syncthreads();
  if (threadIdx.x < s.nrhs) {
    const int r = threadIdx.x;
    const double beta = sqrt(n2s[r]);
    if (first) {
      s.bnorm[r] = beta;
      s.active[r] = beta > 0;
      s.applies[r] = 0;
      s.relres[r] = beta > 0 ? 1.0 : 0.0;
    } else if (s.active[r]) {
      s.applies[r] += 1;
      s.relres[r] = beta / s.bnorm[r];
      if (beta <= s.tol * s.bnorm[r]) s.active[r] = 0;
    }
    s.kcnt[r] = 0;
    double2* gv = s.gv + (long long)r * (s.m + 1);
    for (int i = 0; i <= s.m; ++i) gv[i] = make_double2(0, 0);
    if (s.active[r]) {
      gv[0] = make_double2(beta, 0);
      s.invh[r] = 1.0 / beta;
      atomicOr(&any, 1);
    } else {
      s.invh[r] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && !any) mark_done(s);
}

// Grid of the cooperative k_arnoldi: one CTA per SM (at most solve_nblk(), the partial-sum rows'
// length); 0 when the device cannot hold it resident.  Found once per device.
template <typename CT>
int arnoldi_grid() {
  static int cache[64];
  static bool init = false;
  if (!init) {
    for (int& c : cache) c = -1;
    init = true;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  if (dev >= 64) dev = 63;
  int& g = cache[dev];
  if (g < 0) {
    int per = 0, coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    int per_long = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_arnoldi<CT, ar_ic<CT>(), 4, 4>, AR_T, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_long, k_arnoldi<CT, 2, ar_ulong<CT>(), 1>, AR_T, 0);
    per = std::min(per, per_long);
    g = (coop && per > 0) ? std::min(amg_sm_count(), solve_nblk()) : 0;
  }
  return g;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }
size_t scal_doubles(int nrhs, int m) { return (size_t)nrhs * ((m + 1) * m + 3 * m + 1) * 2 + 3 * (size_t)nrhs; }

template <typename CT>
amg_status solve_impl(amg_coarse* h, long long rows, amg_apply_fn op, const CT* b, CT* x, int nrhs, double tol, int m,
                      int max_applies, cudaStream_t st, double* info, unsigned char* ws, bool poll) {
  const long long vstride = rows * nrhs;
  const bool flat = nrhs > 1 && 32 % nrhs == 0;  // coalesced flat loops (see k_dots_flat)
  const int ar_grid = 32 % nrhs == 0 ? arnoldi_grid<CT>() : 0;  // fused step (k_arnoldi) when > 0
  SolveWork& sw = h->sw;
  FState s;
  s.m = m;
  s.nrhs = nrhs;
  const int nblk = solve_nblk();
  s.nblk = nblk;
  s.rows = rows;
  s.tol = tol;
  unsigned char* p = ws;
  CT* V = (CT*)p;                       // V_0 .. V_m
  CT* cur = V + (size_t)(m + 1) * vstride;  // unnormalised next basis vector (V_j = cur * invh)
  CT* nxt = cur + vstride;                  // D_c V_j, orthogonalised in place
  p += align256((size_t)(m + 3) * vstride * sizeof(CT));
  s.part = (double2*)p;
  p += align256((size_t)(m + 1) * nblk * nrhs * sizeof(double2));
  double2* d2 = (double2*)p;
  s.H = d2;
  d2 += (size_t)nrhs * (m + 1) * m;
  s.cs = d2;
  d2 += (size_t)nrhs * m;
  s.sn = d2;
  d2 += (size_t)nrhs * m;
  s.gv = d2;
  d2 += (size_t)nrhs * (m + 1);
  double* q = (double*)d2;
  s.bnorm = q;
  s.relres = q + nrhs;
  s.invh = q + 2 * nrhs;
  p += align256(scal_doubles(nrhs, m) * sizeof(double));
  int* fl = (int*)p;
  s.active = fl;
  s.kcnt = fl + nrhs;
  s.applies = fl + 2 * nrhs;
  s.done = fl + 3 * nrhs;
  s.counter = (unsigned*)(fl + 3 * nrhs + 4);
  s.bar = (unsigned*)(fl + 3 * nrhs + 5);
  s.err = h->err;
  s.hdone = poll ? sw.hdone_dev : nullptr;
  s.bar_extra = sw.test_extra_arrivals;
  if (poll) sw.ticket = sw.ticket >= (1 << 30) ? 1 : sw.ticket + 1;  // never 0, the word's initial value
  s.ticket = poll ? sw.ticket : 0;
  const unsigned egrid = 4 * amg_sm_count();
  AMG_CUDA_TRY(cudaMemsetAsync(fl, 0, (4 * (size_t)nrhs + 8) * sizeof(int), st));
  k_residual<CT><<<nblk, ST_T, 0, st>>>(s, cur, b, 1, x);  // also x = 0
  AMG_LAUNCH_CHECK();
  h->launches += 1;
  // The kernel that finds every right-hand side converged writes this solve's ticket into the
  // mapped host word.  An event follows each Arnoldi step (and each restart residual); once the
  // next application is queued the host waits for that event and reads the word, so the device
  // always has an application in hand while the host decides, and a converged solve launches no
  // further Arnoldi step (its one speculative application returns at once on the device flag).
  int pending = -1;
  auto record = [&]() {
    if (!poll) return;
    pending = (pending + 1) % SolveWork::kRing;
    cudaEventRecord(sw.ev[pending], st);
  };
  auto converged = [&]() -> bool {
    if (!poll) return false;
    cudaEventSynchronize(sw.ev[pending]);
    return *(volatile int*)sw.hflag == s.ticket;
  };
  record();
  bool stop = false;
  int launched = 0;
  while (launched < max_applies && !stop) {
    const int mc = std::min(m, max_applies - launched);
    for (int j = 0; j < mc; ++j) {
      // V_j = cur / h_{j,j-1} is written by the application itself, which reads cur scaled
      amg_status status = op(h, cur, nxt, nrhs, st, s.done, s.invh, V + j * vstride);
      if (status != AMG_OK) return status;
      ++launched;
      if (converged()) {
        stop = true;
        break;
      }
      if (ar_grid > 0) {
        const CT* Vr = V;
        int jj = j;
        void* args[] = {&s, &nxt, &Vr, (void*)&vstride, &jj};
        const void* kern = rows * nrhs > AR_LONG ? (const void*)k_arnoldi<CT, 2, ar_ulong<CT>(), 1>
                                                 : (const void*)k_arnoldi<CT, ar_ic<CT>(), 4, 4>;
        AMG_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(ar_grid), dim3(AR_T), args, 0, st));
        h->launches += 1;
      } else {
        if (flat) {
          k_dots_flat<CT><<<dim3(nblk, j + 1), ST_T, 0, st>>>(s, nxt, V, vstride, j);
          k_update_flat<CT><<<nblk, ST_T, 0, st>>>(s, nxt, V, vstride, j);
        } else {
          k_dots<CT><<<dim3(nblk, j + 1), ST_T, 0, st>>>(s, nxt, V, vstride, j);
          k_update<CT><<<nblk, ST_T, 0, st>>>(s, nxt, V, vstride, j);
        }
        AMG_LAUNCH_CHECK();
        h->launches += 2;
      }
      std::swap(cur, nxt);
      record();
    }
    k_xupdate<CT><<<egrid, ST_T, 0, st>>>(s, x, V, vstride);
    AMG_LAUNCH_CHECK();
    h->launches += 1;
    if (launched >= max_applies || stop) break;
    amg_status status = op(h, x, cur, nrhs, st, s.done, nullptr, nullptr);
    if (status != AMG_OK) return status;
    ++launched;
    k_residual<CT><<<nblk, ST_T, 0, st>>>(s, cur, b, 0, (CT*)nullptr);
    AMG_LAUNCH_CHECK();
    h->launches += 1;
    record();
  }
  if (info) {
    int applies[MAXR];
    double rel[MAXR];
    AMG_CUDA_TRY(cudaMemcpyAsync(applies, s.applies, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaMemcpyAsync(rel, s.relres, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    for (int r = 0; r < nrhs; ++r) {
      info[2 * r] = applies[r];
      info[2 * r + 1] = rel[r];
    }
  }
  return AMG_OK;
}

}  // namespace

size_t amg_internal_solve_bytes(const amg_coarse* h, int nrhs, int m) {
  const size_t N = (size_t)h->g.Vc * h->g.nc * nrhs * coarse_elem_bytes(h);
  return align256((size_t)(m + 3) * N) + align256((size_t)(m + 1) * solve_nblk() * nrhs * sizeof(double2)) +
         align256(scal_doubles(nrhs, m) * sizeof(double)) + align256((4 * (size_t)nrhs + 8) * sizeof(int));
}

amg_status amg_internal_solve_ws(amg_coarse* h, const void* b, void* x, int nrhs, double tol, int restart,
                                 int max_applies, cudaStream_t s, double* info, void* ws, bool poll) {
  if (nrhs > MAXR || restart < 1 || restart > AMG_MAX_NTV || max_applies < 1) return AMG_ERR_INVALID_ARG;
  const long long rows = h->g.Vc * h->g.nc;
  if (h->p.vec_prec == AMG_FP64)
    return solve_impl<double2>(h, rows, amg_internal_apply_ex, (const double2*)b, (double2*)x, nrhs, tol, restart,
                               max_applies, s, info, (unsigned char*)ws, poll);
  return solve_impl<float2>(h, rows, amg_internal_apply_ex, (const float2*)b, (float2*)x, nrhs, tol, restart,
                            max_applies, s, info, (unsigned char*)ws, poll);
}

namespace {
amg_status ensure_solve_work(amg_coarse* h, int nrhs, int restart, cudaStream_t s) {
  SolveWork& sw = h->sw;
  const size_t need = amg_internal_solve_bytes(h, nrhs, restart);
  if (need > sw.bytes) {
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(sw.buf);
    sw.buf = nullptr;
    sw.bytes = 0;
    AMG_CUDA_TRY(cudaMalloc(&sw.buf, need));
    sw.bytes = need;
  }
  if (!sw.hflag) {
    AMG_CUDA_TRY(cudaHostAlloc((void**)&sw.hflag, sizeof(int), cudaHostAllocMapped));
    *sw.hflag = 0;
    AMG_CUDA_TRY(cudaHostGetDevicePointer((void**)&sw.hdone_dev, sw.hflag, 0));
    for (int k = 0; k < SolveWork::kRing; ++k)
      AMG_CUDA_TRY(cudaEventCreateWithFlags(&sw.ev[k], cudaEventDisableTiming));
  }
  return AMG_OK;
}
}  // namespace

amg_status amg_internal_solve_op(amg_coarse* h, long long rows, amg_apply_fn op, const void* b, void* x, int nrhs,
                                 double tol, int restart, int max_applies, cudaStream_t s, double* info) {
  if (nrhs > MAXR || restart < 1 || restart > AMG_MAX_NTV || max_applies < 1) return AMG_ERR_INVALID_ARG;
  if (rows > h->g.Vc * h->g.nc) return AMG_ERR_INVALID_ARG;  // the workspace is sized for D_c's rows
  amg_status st = ensure_solve_work(h, nrhs, restart, s);
  if (st != AMG_OK) return st;
  unsigned char* ws = (unsigned char*)h->sw.buf;
  if (h->p.vec_prec == AMG_FP64)
    return solve_impl<double2>(h, rows, op, (const double2*)b, (double2*)x, nrhs, tol, restart, max_applies, s,
                               info, ws, true);
  return solve_impl<float2>(h, rows, op, (const float2*)b, (float2*)x, nrhs, tol, restart, max_applies, s, info,
                            ws, true);
}

amg_status amg_internal_solve(amg_coarse* h, const void* b, void* x, int nrhs, double tol, int restart,
                              int max_applies, cudaStream_t s, double* info) {
  if (nrhs > MAXR || restart < 1 || restart > AMG_MAX_NTV || max_applies < 1) return AMG_ERR_INVALID_ARG;
  AMG_TRY_INTERNAL(ensure_solve_work(h, nrhs, restart, s));
  return amg_internal_solve_ws(h, b, x, nrhs, tol, restart, max_applies, s, info, h->sw.buf, true);
}

extern "C" amg_status amg_grid_cap_test_hook(amg_handle h, int max_ctas) {
  if (!h || max_ctas < 0) return AMG_ERR_INVALID_ARG;
  h->grid_cap = max_ctas;
  return AMG_OK;
}

extern "C" amg_status amg_solve_test_hook(amg_handle h, int extra_arrivals) {
  if (!h || extra_arrivals < 0) return AMG_ERR_INVALID_ARG;
  h->sw.test_extra_arrivals = (unsigned)extra_arrivals;
  return AMG_OK;
}
