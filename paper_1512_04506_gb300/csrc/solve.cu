// Coarse-grid solve of Alg. 2: restarted FGMRES(m) on D_c with classical Gram-Schmidt Arnoldi
// ("BLAS-like linear algebra (mainly Gram-Schmidt)") and Givens rotations, one independent
// Krylov space per right-hand side.  Vectors stay in the coarse layout [Vc][2][ntv][nrhs]; all
// scalars (Hessenberg matrix, rotations, residual estimates, convergence flags) live on the
// device, so the host only launches kernels.  Once every right-hand side has converged the
// device flag `done` makes all later kernels of the iteration return immediately; the host
// learns of it through an event two iterations behind the launch front, so the GPU never waits
// for the host.
#include "amg_internal.cuh"

#include <algorithm>

namespace {

constexpr int ST_T = 256;
constexpr int MAXR = 16;

struct FState {
  int m, nrhs, nblk;
  long long rows;  // Vc * nc
  double tol;
  double2 *H, *cs, *sn, *gv, *yv, *part;
  double *bnorm, *relres, *invh;
  int *active, *kcnt, *applies, *done;
};

__device__ inline double2 to_d(float2 v) { return make_double2(v.x, v.y); }
__device__ inline double2 to_d(double2 v) { return v; }
template <typename CT> __device__ inline CT from_d(double2 v);
template <> __device__ inline float2 from_d<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ inline double2 from_d<double2>(double2 v) { return v; }

// CTA-wide sum of nrhs complex values per thread; result written by thread r < nrhs to out[r].
__device__ inline void cta_sum_store(double2 (&acc)[MAXR], int nrhs, double2* out, int stride) {
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
    out[threadIdx.x * stride] = t;
  }
}

// part[(i * nblk + b) * nrhs + r] = partial <V_i, w> (i = blockIdx.y).
template <typename CT>
__global__ void __launch_bounds__(ST_T) k_dots(FState s, const CT* __restrict__ w, const CT* __restrict__ V,
                                               long long vstride) {
  if (*s.done) return;
  const int i = blockIdx.y;
  const CT* Vi = V + i * vstride;
  // per-thread sums in the vector precision, CTA and grid sums in FP64
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
  cta_sum_store(acc, s.nrhs, s.part + ((long long)i * s.nblk + blockIdx.x) * s.nrhs, 1);
}

// H[r][i][j] = sum of the partial dots (zero for converged right-hand sides).
__global__ void k_finish_dots(FState s, int j) {
  const int t = threadIdx.x + blockIdx.x * blockDim.x;
  if (*s.done || t >= (j + 1) * s.nrhs) return;
  const int i = t / s.nrhs, r = t % s.nrhs;
  double2 sum = make_double2(0, 0);
  for (int b = 0; b < s.nblk; ++b) sum = cadd(sum, s.part[((long long)i * s.nblk + b) * s.nrhs + r]);
  s.H[((long long)r * (s.m + 1) + i) * s.m + j] = s.active[r] ? sum : make_double2(0, 0);
}

// w -= sum_{i<=j} H[r][i][j] V_i; partial |w|^2 into part slot 0.
template <typename CT>
__global__ void __launch_bounds__(ST_T) k_update(FState s, CT* __restrict__ w, const CT* __restrict__ V,
                                                 long long vstride, int j) {
  if (*s.done) return;
  __shared__ CT hc[AMG_MAX_NTV + 1][MAXR];
  for (int e = threadIdx.x; e < (j + 1) * s.nrhs; e += ST_T) {
    const int i = e / s.nrhs, r = e % s.nrhs;
    hc[i][r] = from_d<CT>(s.H[((long long)r * (s.m + 1) + i) * s.m + j]);
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
  cta_sum_store(acc, s.nrhs, s.part + (long long)blockIdx.x * s.nrhs, 1);
}

// One thread per right-hand side: h_{j+1,j}, Givens rotations, residual estimate, convergence.
__global__ void k_arnoldi(FState s, int j) {
  __shared__ int any;
  if (*s.done) return;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int r = threadIdx.x;
  if (r < s.nrhs) {
    if (s.active[r]) {
      double n2 = 0;
      for (int b = 0; b < s.nblk; ++b) n2 += s.part[(long long)b * s.nrhs + r].x;
      const double hnext = sqrt(n2);
      double2* Hc = s.H + (long long)r * (s.m + 1) * s.m;  // Hc[i * m + j]
      double2* cs = s.cs + (long long)r * s.m;
      double2* sn = s.sn + (long long)r * s.m;
      double2* gv = s.gv + (long long)r * (s.m + 1);
      Hc[(j + 1) * s.m + j] = make_double2(hnext, 0);
      for (int i = 0; i < j; ++i) {
        const double2 a = Hc[i * s.m + j], b = Hc[(i + 1) * s.m + j];
        const double2 t = cadd(cmul(cs[i], a), cmul(sn[i], b));
        Hc[(i + 1) * s.m + j] = csub(cmul(cconj(cs[i]), b), cmul(cconj(sn[i]), a));
        Hc[i * s.m + j] = t;
      }
      const double2 a = Hc[j * s.m + j];
      const double den = sqrt(a.x * a.x + a.y * a.y + hnext * hnext);
      const double2 c = den > 0 ? cscale(cconj(a), 1.0 / den) : make_double2(1, 0);
      const double2 sv = den > 0 ? make_double2(hnext / den, 0) : make_double2(0, 0);
      cs[j] = c;
      sn[j] = sv;
      Hc[j * s.m + j] = make_double2(den, 0);
      Hc[(j + 1) * s.m + j] = make_double2(0, 0);
      const double2 gj = gv[j];
      gv[j + 1] = cscale(cmul(cconj(sv), gj), -1.0);
      gv[j] = cmul(c, gj);
      const double rel = sqrt(gv[j + 1].x * gv[j + 1].x + gv[j + 1].y * gv[j + 1].y) / s.bnorm[r];
      s.relres[r] = rel;
      s.kcnt[r] = j + 1;
      s.applies[r] += 1;
      if (rel <= s.tol || hnext == 0) {
        s.active[r] = 0;
        s.invh[r] = 0;
      } else {
        s.invh[r] = 1.0 / hnext;
        atomicOr(&any, 1);
      }
    } else {
      s.invh[r] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && !any) *s.done = 1;
}

// out = w * invh[r]
template <typename CT>
__global__ void k_scale(FState s, CT* __restrict__ out, const CT* __restrict__ w) {
  if (*s.done) return;
  const long long n = s.rows * s.nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const CT v = w[e];
    const auto f = (decltype(v.x))s.invh[e % s.nrhs];
    out[e] = CT{v.x * f, v.y * f};
  }
}

// Back substitution of the k x k triangular system per right-hand side.
__global__ void k_backsolve(FState s) {
  const int r = threadIdx.x;
  if (r >= s.nrhs) return;
  const int k = s.kcnt[r];
  const double2* Hc = s.H + (long long)r * (s.m + 1) * s.m;
  const double2* gv = s.gv + (long long)r * (s.m + 1);
  double2* y = s.yv + (long long)r * s.m;
  for (int i = k - 1; i >= 0; --i) {
    double2 t = gv[i];
    for (int l = i + 1; l < k; ++l) t = csub(t, cmul(Hc[i * s.m + l], y[l]));
    const double2 d = Hc[i * s.m + i];
    const double dd = d.x * d.x + d.y * d.y;
    y[i] = dd > 0 ? cscale(cmulc(d, t), 1.0 / dd) : make_double2(0, 0);
  }
  for (int i = k; i < s.m; ++i) y[i] = make_double2(0, 0);
}

// x += sum_i y[r][i] V_i (over the columns built in this cycle); kcnt is then reset.
template <typename CT>
__global__ void k_xupdate(FState s, CT* __restrict__ x, const CT* __restrict__ V, long long vstride) {
  __shared__ CT yc[AMG_MAX_NTV][MAXR];
  __shared__ int kmax;
  if (threadIdx.x == 0) {
    int k = 0;
    for (int r = 0; r < s.nrhs; ++r) k = max(k, s.kcnt[r]);
    kmax = k;
  }
  for (int e = threadIdx.x; e < s.m * s.nrhs; e += blockDim.x) {
    const int i = e / s.nrhs, r = e % s.nrhs;
    yc[i][r] = from_d<CT>(s.yv[(long long)r * s.m + i]);
  }
  __syncthreads();
  const long long n = s.rows * s.nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % s.nrhs);
    CT v = x[e];
    for (int i = 0; i < kmax; ++i) {
      const CT q = V[i * vstride + e];
      const CT c = yc[i][r];
      v.x += c.x * q.x - c.y * q.y;
      v.y += c.x * q.y + c.y * q.x;
    }
    x[e] = v;
  }
}

// w = b - w (restart residual; first = 1: w = b) and partial |w|^2.
template <typename CT>
__global__ void __launch_bounds__(ST_T) k_residual(FState s, CT* __restrict__ w, const CT* __restrict__ b, int first) {
  if (*s.done) return;
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
        const CT a = w[row * s.nrhs + r];
        v.x -= a.x;
        v.y -= a.y;
      }
      w[row * s.nrhs + r] = v;
      a[r].x += v.x * v.x + v.y * v.y;
    }
  }
  double2 acc[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) acc[r] = to_d(a[r]);
  cta_sum_store(acc, s.nrhs, s.part + (long long)blockIdx.x * s.nrhs, 1);
}

// Start of a restart cycle: beta = |r|, convergence check, g = (beta, 0, ...), invh = 1/beta.
__global__ void k_start(FState s, int first) {
  __shared__ int any;
  if (*s.done) return;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int r = threadIdx.x;
  if (r < s.nrhs) {
    double n2 = 0;
    for (int b = 0; b < s.nblk; ++b) n2 += s.part[(long long)b * s.nrhs + r].x;
    const double beta = sqrt(n2);
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
  if (threadIdx.x == 0 && !any) *s.done = 1;
}

template <typename CT>
amg_status solve_impl(amg_coarse* h, const CT* b, CT* x, int nrhs, double tol, int m, int max_applies,
                      cudaStream_t st, double* info) {
  const Geom& g = h->g;
  const long long rows = g.Vc * g.nc;
  const long long vstride = rows * nrhs;
  SolveWork& sw = h->sw;
  const int nblk = 2 * 152;
  if (sw.nrhs != nrhs || sw.restart != m) {
    cudaStreamSynchronize(st);
    cudaFree(sw.basis);
    cudaFree(sw.w);
    cudaFree(sw.part);
    cudaFree(sw.scal);
    cudaFree(sw.flags);
    sw = SolveWork();
    AMG_CUDA_TRY(cudaMalloc(&sw.basis, (size_t)(m + 1) * vstride * sizeof(CT)));
    AMG_CUDA_TRY(cudaMalloc(&sw.w, (size_t)vstride * sizeof(CT)));
    AMG_CUDA_TRY(cudaMalloc(&sw.part, (size_t)(m + 1) * nblk * nrhs * sizeof(double2)));
    const size_t nscal = (size_t)nrhs * ((m + 1) * m + 2 * m + (m + 1) + m) * 2 + 4 * nrhs;
    AMG_CUDA_TRY(cudaMalloc(&sw.scal, nscal * sizeof(double)));
    AMG_CUDA_TRY(cudaMalloc(&sw.flags, (size_t)(3 * nrhs + 1) * sizeof(int)));
    sw.nrhs = nrhs;
    sw.restart = m;
  }
  FState s;
  s.m = m;
  s.nrhs = nrhs;
  s.nblk = nblk;
  s.rows = rows;
  s.tol = tol;
  double2* p = (double2*)sw.scal;
  s.H = p;
  p += (size_t)nrhs * (m + 1) * m;
  s.cs = p;
  p += (size_t)nrhs * m;
  s.sn = p;
  p += (size_t)nrhs * m;
  s.gv = p;
  p += (size_t)nrhs * (m + 1);
  s.yv = p;
  p += (size_t)nrhs * m;
  double* q = (double*)p;
  s.bnorm = q;
  s.relres = q + nrhs;
  s.invh = q + 2 * nrhs;
  s.part = sw.part;
  s.active = sw.flags;
  s.kcnt = sw.flags + nrhs;
  s.applies = sw.flags + 2 * nrhs;
  s.done = sw.flags + 3 * nrhs;
  CT* V = (CT*)sw.basis;
  CT* w = (CT*)sw.w;
  const unsigned egrid = 4 * 152;
  AMG_CUDA_TRY(cudaMemsetAsync(s.done, 0, sizeof(int), st));
  AMG_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)vstride * sizeof(CT), st));
  k_residual<CT><<<nblk, ST_T, 0, st>>>(s, w, b, 1);
  h->launches++;
  k_start<<<1, 64, 0, st>>>(s, 1);
  h->launches++;
  k_scale<CT><<<egrid, 256, 0, st>>>(s, V, w);
  h->launches++;
  AMG_LAUNCH_CHECK();
  // host-side view of `done`, two iterations behind the launch front
  int* hflag = nullptr;
  AMG_CUDA_TRY(cudaHostAlloc((void**)&hflag, 64 * sizeof(int), cudaHostAllocDefault));
  cudaEvent_t ev[64];
  for (int k = 0; k < 64; ++k) cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
  int launched = 0, polled = 0, issued = 0;
  bool stop = false;
  auto poll_point = [&]() -> void {
    const int slot = issued % 64;
    cudaMemcpyAsync(hflag + slot, s.done, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaEventRecord(ev[slot], st);
    ++issued;
    while (issued - polled > 2) {
      const int ps = polled % 64;
      cudaEventSynchronize(ev[ps]);
      if (hflag[ps]) stop = true;
      ++polled;
    }
  };
  amg_status status = AMG_OK;
  while (launched < max_applies && !stop) {
    const int mc = std::min(m, max_applies - launched);
    for (int j = 0; j < mc && !stop; ++j) {
      status = amg_internal_apply_ex(h, V + j * vstride, w, nrhs, st, s.done);
      if (status != AMG_OK) break;
      k_dots<CT><<<dim3(nblk, j + 1), ST_T, 0, st>>>(s, w, V, vstride);
      h->launches++;
      k_finish_dots<<<((j + 1) * nrhs + 127) / 128, 128, 0, st>>>(s, j);
      h->launches++;
      k_update<CT><<<nblk, ST_T, 0, st>>>(s, w, V, vstride, j);
      h->launches++;
      k_arnoldi<<<1, 64, 0, st>>>(s, j);
      h->launches++;
      k_scale<CT><<<egrid, 256, 0, st>>>(s, V + (j + 1) * vstride, w);
      h->launches++;
      ++launched;
      poll_point();
    }
    if (status != AMG_OK) break;
    k_backsolve<<<1, 64, 0, st>>>(s);
    h->launches++;
    k_xupdate<CT><<<egrid, 256, 0, st>>>(s, x, V, vstride);
    h->launches++;
    if (launched >= max_applies || stop) break;
    status = amg_internal_apply_ex(h, x, w, nrhs, st, s.done);
    if (status != AMG_OK) break;
    ++launched;
    k_residual<CT><<<nblk, ST_T, 0, st>>>(s, w, b, 0);
    h->launches++;
    k_start<<<1, 64, 0, st>>>(s, 0);
    h->launches++;
    k_scale<CT><<<egrid, 256, 0, st>>>(s, V, w);
    h->launches++;
    poll_point();
  }
  cudaError_t le = cudaGetLastError();
  cudaStreamSynchronize(st);
  for (int k = 0; k < 64; ++k) cudaEventDestroy(ev[k]);
  cudaFreeHost(hflag);
  if (status != AMG_OK) return status;
  if (le != cudaSuccess) return AMG_ERR_CUDA;
  if (info) {
    int applies[MAXR];
    double rel[MAXR];
    AMG_CUDA_TRY(cudaMemcpy(applies, s.applies, nrhs * sizeof(int), cudaMemcpyDeviceToHost));
    AMG_CUDA_TRY(cudaMemcpy(rel, s.relres, nrhs * sizeof(double), cudaMemcpyDeviceToHost));
    for (int r = 0; r < nrhs; ++r) {
      info[2 * r] = applies[r];
      info[2 * r + 1] = rel[r];
    }
  }
  return AMG_OK;
}

}  // namespace

amg_status amg_internal_solve(amg_coarse* h, const void* b, void* x, int nrhs, double tol, int restart,
                              int max_applies, cudaStream_t s, double* info) {
  if (nrhs > MAXR || restart < 1 || restart > AMG_MAX_NTV || max_applies < 1) return AMG_ERR_INVALID_ARG;
  if (h->p.vec_prec == AMG_FP64)
    return solve_impl<double2>(h, (const double2*)b, (double2*)x, nrhs, tol, restart, max_applies, s, info);
  return solve_impl<float2>(h, (const float2*)b, (float2*)x, nrhs, tol, restart, max_applies, s, info);
}
