// Mixed-precision coarse solve: iterative refinement around the low-precision FGMRES of Alg. 2.
//
// The paper keeps D_c in half precision inside a coarse solve that only needs a residual of about
// 0.05 (Sec. 3).  To reach a tighter coarse tolerance with the cheap operator, each pass solves the
// correction equation D_c e = r with FGMRES on the FP16 / BF16 operator (handle h_inner) to
// inner_tol, adds e to x, and recomputes the true residual r = b - D_c x with the accurate FP32
// operator (handle h_outer); right-hand sides that have reached tol drop out (their r is zeroed,
// so the inner solver leaves them alone).
#include "amg_internal.cuh"

#include <cmath>
#include <vector>

namespace {

// per right-hand side |v_r|^2 of a coarse FP32 vector [rows][nrhs]: a grid-stride pass over the
// rows with coalesced reads, four elements' loads issued together.  When the stride is a multiple
// of nrhs (nrhs = 1, 2, 4, 8, 16) a thread only meets column e % nrhs: its partial sum stays in
// FP32 (a few dozen terms) and is summed over the lanes of equal column in FP32, over the warps
// and CTAs in FP64 (one double atomicAdd per CTA and column into out, zeroed by the caller).
// Other column counts keep one FP64 partial per column.
__global__ void __launch_bounds__(256) k_colnorm2(const float2* __restrict__ v, long long rows, int nrhs,
                                                  double* __restrict__ out) {
  __shared__ double red[16][8];
  const long long n = rows * nrhs;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (stride % nrhs == 0 && 32 % nrhs == 0) {
    float s = 0.f;
    for (long long eb = e0; eb < n; eb += 4 * stride) {
      float2 a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = eb + u * stride < n ? v[eb + u * stride] : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 4; ++u) s += a[u].x * a[u].x + a[u].y * a[u].y;
    }
    for (int o = 16; o >= nrhs; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane < nrhs) red[lane][warp] = (double)s;
  } else {
    double acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] = 0.0;
    for (long long e = e0; e < n; e += stride) {
      const float2 a = v[e];
      const double q = (double)a.x * a.x + (double)a.y * a.y;
#pragma unroll
      for (int r = 0; r < 16; ++r)
        if (r == (int)(e % nrhs)) acc[r] += q;
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (r >= nrhs) break;
      double t = acc[r];
      for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) red[r][warp] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    atomicAdd(out + threadIdx.x, t);
  }
}

// x += e; r = b - w (w = D_c x from the accurate operator), columns with keep[r] == 0 zeroed in r;
// four elements' loads per round
__global__ void k_axpy(float2* __restrict__ x, const float2* __restrict__ e, long long n) {
  const long long es = (long long)gridDim.x * blockDim.x;
  for (long long ib = blockIdx.x * (long long)blockDim.x + threadIdx.x; ib < n; ib += 4 * es) {
    float2 a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long i = ib + u * es;
      a[u] = i < n ? x[i] : make_float2(0.f, 0.f);
      b[u] = i < n ? e[i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (ib + u * es < n) x[ib + u * es] = make_float2(a[u].x + b[u].x, a[u].y + b[u].y);
  }
}
__global__ void k_resid(float2* __restrict__ r, const float2* __restrict__ b, const float2* __restrict__ w,
                        const int* __restrict__ keep, long long n, int nrhs) {
  const long long es = (long long)gridDim.x * blockDim.x;
  for (long long ib = blockIdx.x * (long long)blockDim.x + threadIdx.x; ib < n; ib += 4 * es) {
    float2 u[4], v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long i = ib + k * es;
      u[k] = i < n ? b[i] : make_float2(0.f, 0.f);
      v[k] = i < n ? w[i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long i = ib + k * es;
      if (i < n) r[i] = keep[i % nrhs] ? make_float2(u[k].x - v[k].x, u[k].y - v[k].y) : make_float2(0.f, 0.f);
    }
  }
}

}  // namespace

extern "C" amg_status amg_coarse_solve_mixed(amg_handle ho, amg_handle hi, const void* d_b, void* d_x, int nrhs,
                                             double tol, double inner_tol, int restart, int max_inner_applies,
                                             int max_outer, void* stream, double* info) {
  if (!ho || !hi || !d_b || !d_x || d_b == d_x || !aligned16(d_b) || !aligned16(d_x)) return AMG_ERR_INVALID_ARG;
  if (nrhs < 1 || nrhs > 16 || nrhs > ho->p.max_nrhs || nrhs > hi->p.max_nrhs) return AMG_ERR_INVALID_ARG;
  if (!(tol > 0) || !(inner_tol > 0) || max_outer < 1 || max_inner_applies < 1) return AMG_ERR_INVALID_ARG;
  if (ho->p.vec_prec == AMG_FP64 || hi->p.vec_prec == AMG_FP64) return AMG_ERR_UNSUPPORTED;
  for (int mu = 0; mu < 4; ++mu)
    if (ho->g.L[mu] != hi->g.L[mu] || ho->g.B[mu] != hi->g.B[mu]) return AMG_ERR_INVALID_ARG;
  if (ho->g.ntv != hi->g.ntv) return AMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ho->last_stream = hi->last_stream = st;
  const long long rows = ho->g.Vc * ho->g.nc, n = rows * nrhs;
  const size_t bytes = (size_t)n * sizeof(float2);
  // workspace: r, e, w (3 coarse vectors) + norms + keep flags, owned by the outer handle
  const size_t need = 3 * bytes + 64 * sizeof(double) + 64 * sizeof(int);
  if (need > ho->tmp_bytes) {
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(ho->xc_tmp);
    cudaFree(ho->yc_tmp);
    ho->xc_tmp = ho->yc_tmp = nullptr;
    ho->tmp_bytes = 0;
    AMG_CUDA_TRY(cudaMalloc(&ho->xc_tmp, need));
    AMG_CUDA_TRY(cudaMalloc(&ho->yc_tmp, need));
    ho->tmp_bytes = need;
  }
  float2* r = (float2*)ho->xc_tmp;
  float2* e = r + n;
  float2* w = e + n;
  double* nrm = (double*)(w + n);
  int* keep = (int*)(nrm + 64);
  const float2* b = (const float2*)d_b;
  float2* x = (float2*)d_x;
  AMG_CUDA_TRY(cudaMemsetAsync(x, 0, bytes, st));
  AMG_CUDA_TRY(cudaMemcpyAsync(r, b, bytes, cudaMemcpyDeviceToDevice, st));
  std::vector<double> bn(nrhs), rn(nrhs), inner(nrhs, 0.0), outer(nrhs, 0.0);
  std::vector<int> kp(nrhs, 1);
  std::vector<double> sub(2 * nrhs);
  AMG_CUDA_TRY(cudaMemsetAsync(nrm, 0, nrhs * sizeof(double), st));
  k_colnorm2<<<2 * amg_sm_count(), 256, 0, st>>>(b, rows, nrhs, nrm);
  AMG_LAUNCH_CHECK();
  ho->launches++;
  AMG_CUDA_TRY(cudaMemcpyAsync(bn.data(), nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  for (int q = 0; q < nrhs; ++q) rn[q] = 1.0;
  for (int it = 0; it < max_outer; ++it) {
    bool all = true;
    for (int q = 0; q < nrhs; ++q) {
      kp[q] = bn[q] > 0 && rn[q] > tol;
      all = all && !kp[q];
    }
    if (all) break;
    if (it > 0) {  // zero the columns that have converged so the inner solve skips them
      AMG_CUDA_TRY(cudaMemcpyAsync(keep, kp.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
      k_resid<<<4 * amg_sm_count(), 256, 0, st>>>(r, b, w, keep, n, nrhs);
      AMG_LAUNCH_CHECK();
      ho->launches++;
    }
    amg_status s = amg_internal_solve(hi, r, e, nrhs, inner_tol, restart, max_inner_applies, st, sub.data());
    if (s != AMG_OK) return s;
    for (int q = 0; q < nrhs; ++q) inner[q] += kp[q] ? sub[2 * q] : 0;
    k_axpy<<<4 * amg_sm_count(), 256, 0, st>>>(x, e, n);
    AMG_LAUNCH_CHECK();
    ho->launches++;
    s = amg_internal_apply(ho, x, w, nrhs, st);
    if (s != AMG_OK) return s;
    for (int q = 0; q < nrhs; ++q) kp[q] = 1;
    AMG_CUDA_TRY(cudaMemcpyAsync(keep, kp.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
    k_resid<<<4 * amg_sm_count(), 256, 0, st>>>(r, b, w, keep, n, nrhs);
    AMG_CUDA_TRY(cudaMemsetAsync(nrm, 0, nrhs * sizeof(double), st));
    k_colnorm2<<<2 * amg_sm_count(), 256, 0, st>>>(r, rows, nrhs, nrm);
    AMG_LAUNCH_CHECK();
    ho->launches += 2;
    AMG_CUDA_TRY(cudaMemcpyAsync(rn.data(), nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    for (int q = 0; q < nrhs; ++q) {
      rn[q] = bn[q] > 0 ? std::sqrt(rn[q] / bn[q]) : 0.0;
      outer[q] += 1;
    }
  }
  if (info)
    for (int q = 0; q < nrhs; ++q) {
      info[3 * q] = inner[q];
      info[3 * q + 1] = outer[q];
      info[3 * q + 2] = rn[q];
    }
  return AMG_OK;
}
