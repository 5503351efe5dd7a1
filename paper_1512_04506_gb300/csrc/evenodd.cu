// Even/odd-reduced coarse solve (Alg. 2: the coarse system is solved by FGMRES "with even/odd
// preconditioning").
//
// D_c couples a coarse site only to itself and its eight neighbours, so on a coarse lattice with
// all extents even the checkerboard halves (parity (x + y + z + t) mod 2) are not coupled inside a
// half.  Eliminating the odd half leaves the Schur complement S = D_ee - D_eo D_oo^-1 D_oe on the
// even sites; FGMRES solves S x_e = b_e - D_eo D_oo^-1 b_o and x_o = D_oo^-1 (b_o - D_oe x_e)
// follows.  One application of S is two streaming passes over half the sites each
// (eo_apply_kernel in stream.cu): w_o = D_oo^-1 D_oe x_e (8 hop blocks and the stored inverse per
// odd site), y_e = D_ee x_e - D_eo w_o (self block + 8 hop blocks per even site), i.e. about the
// bytes of one application of D_c.
//
// Half vectors [Vc/2][2 ntv][nrhs] list the sites of one parity in lexicographic order: with an
// even x extent the site i of either parity is entry i / 2 of its half.
//
// Setup (amg_setup_evenodd): the inverse of every odd site's self block D_c[i][0], by
// Gauss-Jordan elimination with partial pivoting in FP64, one CTA per site, stored in FP64
// (export) and in the apply precision (layout of D_c's apply copy).
#include "amg_internal.cuh"

#include <vector>

namespace {

constexpr int kSlots = 6;  // half vectors: z_o, w_o, b_e, b_o, reduced rhs, x_e

// Gauss-Jordan inverse of A = D_c[site][0] (row-major FP64) for the odd site of half index h.
__global__ void __launch_bounds__(256) self_inverse_kernel(const double2* __restrict__ Dc64,
                                                           const int* __restrict__ site_of, int nc,
                                                           double2* __restrict__ inv64, void* __restrict__ invq,
                                                           int q_fp64, unsigned* err) {
  extern __shared__ double2 smd[];
  double2* A = smd;             // [nc][nc]
  double2* Bm = smd + nc * nc;  // [nc][nc], starts as the identity
  double2* col = Bm + nc * nc;  // [nc] elimination factors
  __shared__ double bestv[8];
  __shared__ int besti[8];
  __shared__ int piv_s;
  const long long h = blockIdx.x;
  const long long site = site_of[h];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const double2* src = Dc64 + site * 9LL * nc * nc;  // direction 0
  for (int e = tid; e < nc * nc; e += nt) {
    A[e] = src[e];
    Bm[e] = make_double2((e / nc) == (e % nc) ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < nc; ++k) {
    // partial pivoting: the row r >= k with the largest |A[r][k]|
    double v = -1.0;
    int vi = k;
    for (int r = k + tid; r < nc; r += nt) {
      const double2 a = A[r * nc + k];
      const double m = a.x * a.x + a.y * a.y;
      if (m > v) {
        v = m;
        vi = r;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, vi, o);
      if (ov > v || (ov == v && oi < vi)) {
        v = ov;
        vi = oi;
      }
    }
    if (lane == 0) {
      bestv[warp] = v;
      besti[warp] = vi;
    }
    __syncthreads();
    if (tid == 0) {
      double bv = bestv[0];
      int bi = besti[0];
      for (int w = 1; w < nt / 32; ++w)
        if (bestv[w] > bv || (bestv[w] == bv && besti[w] < bi)) {
          bv = bestv[w];
          bi = besti[w];
        }
      piv_s = bi;
      if (!(bv > 0.0) || !isfinite(bv)) atomicOr(err, AMG_EBIT_NONFINITE);  // singular self block
    }
    __syncthreads();
    const int p = piv_s;
    if (p != k)
      for (int c = tid; c < nc; c += nt) {
        const double2 t0 = A[k * nc + c], t1 = Bm[k * nc + c];
        A[k * nc + c] = A[p * nc + c];
        Bm[k * nc + c] = Bm[p * nc + c];
        A[p * nc + c] = t0;
        Bm[p * nc + c] = t1;
      }
    __syncthreads();
    const double2 pk = A[k * nc + k];
    const double den = pk.x * pk.x + pk.y * pk.y;
    const double2 ip = make_double2(pk.x / den, -pk.y / den);
    __syncthreads();
    for (int c = tid; c < nc; c += nt) {
      A[k * nc + c] = cmul(A[k * nc + c], ip);
      Bm[k * nc + c] = cmul(Bm[k * nc + c], ip);
    }
    __syncthreads();
    for (int r = tid; r < nc; r += nt) col[r] = r == k ? make_double2(0, 0) : A[r * nc + k];
    __syncthreads();
    for (int e = tid; e < nc * nc; e += nt) {
      const int r = e / nc, c = e % nc;
      const double2 f = col[r];
      const double2 ak = A[k * nc + c], bk = Bm[k * nc + c];
      A[e] = make_double2(A[e].x - (f.x * ak.x - f.y * ak.y), A[e].y - (f.x * ak.y + f.y * ak.x));
      Bm[e] = make_double2(Bm[e].x - (f.x * bk.x - f.y * bk.y), Bm[e].y - (f.x * bk.y + f.y * bk.x));
    }
    __syncthreads();
  }
  // Bm = A^-1: FP64 row-major copy, and the apply copy column-major [col][row]
  for (int e = tid; e < nc * nc; e += nt) {
    const int r = e / nc, c = e % nc;
    const double2 v = Bm[e];
    inv64[h * nc * nc + e] = v;
    const long long qi = h * nc * nc + (long long)c * nc + r;
    if (q_fp64) reinterpret_cast<double2*>(invq)[qi] = v;
    else reinterpret_cast<float2*>(invq)[qi] = make_float2((float)v.x, (float)v.y);
  }
}

// full [Vc][nc][nrhs] <-> halves [Vc/2][nc][nrhs]
template <typename CT>
__global__ void eo_split_kernel(const CT* __restrict__ v, CT* __restrict__ ve, CT* __restrict__ vo, const Geom g,
                                int nrhs) {
  const long long per = (long long)g.nc * nrhs, total = g.Vc * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / per, rest = e % per;
    const int par = (int)((i % g.Lc[0] + (i / g.Lc[0]) % g.Lc[1] + (i / ((long long)g.Lc[0] * g.Lc[1])) % g.Lc[2] +
                           i / ((long long)g.Lc[0] * g.Lc[1] * g.Lc[2])) & 1);
    (par ? vo : ve)[(i >> 1) * per + rest] = v[e];
  }
}
template <typename CT>
__global__ void eo_merge_kernel(const CT* __restrict__ ve, const CT* __restrict__ vo, CT* __restrict__ v, const Geom g,
                                int nrhs) {
  const long long per = (long long)g.nc * nrhs, total = g.Vc * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / per, rest = e % per;
    const int par = (int)((i % g.Lc[0] + (i / g.Lc[0]) % g.Lc[1] + (i / ((long long)g.Lc[0] * g.Lc[1])) % g.Lc[2] +
                           i / ((long long)g.Lc[0] * g.Lc[1] * g.Lc[2])) & 1);
    v[e] = (par ? vo : ve)[(i >> 1) * per + rest];
  }
}

size_t half_bytes(const amg_coarse* h, int nrhs) {
  return ((size_t)(h->g.Vc / 2) * h->g.nc * nrhs * coarse_elem_bytes(h) + 255) / 256 * 256;
}
void* slot(amg_coarse* h, int k, int nrhs) { return (unsigned char*)h->eo_tmp + (size_t)k * half_bytes(h, nrhs); }

amg_status split_merge(amg_coarse* h, bool split, const void* a, void* b, void* c, int nrhs, cudaStream_t st) {
  if (h->p.vec_prec == AMG_FP64) {
    if (split) eo_split_kernel<double2><<<4 * amg_sm_count(), 256, 0, st>>>((const double2*)a, (double2*)b, (double2*)c, h->g, nrhs);
    else eo_merge_kernel<double2><<<4 * amg_sm_count(), 256, 0, st>>>((const double2*)a, (const double2*)b, (double2*)c, h->g, nrhs);
  } else {
    if (split) eo_split_kernel<float2><<<4 * amg_sm_count(), 256, 0, st>>>((const float2*)a, (float2*)b, (float2*)c, h->g, nrhs);
    else eo_merge_kernel<float2><<<4 * amg_sm_count(), 256, 0, st>>>((const float2*)a, (const float2*)b, (float2*)c, h->g, nrhs);
  }
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

bool eo_ready(const amg_coarse* h) { return h && h->Dinvq && h->eo_site && h->eo_tmp; }

amg_status check_eo_vec(amg_coarse* h, const void* a, const void* b, int nrhs) {
  if (!h || !a || !b || a == b || !aligned16(a) || !aligned16(b)) return AMG_ERR_INVALID_ARG;
  if (nrhs < 1 || nrhs > 16 || nrhs > h->p.max_nrhs) return AMG_ERR_INVALID_ARG;
  if (!eo_ready(h)) return AMG_ERR_UNSUPPORTED;
  return AMG_OK;
}

// x = solution of D_c x = b (full coarse vectors) through the even/odd reduction.
amg_status eo_solve(amg_coarse* h, const void* b, void* x, int nrhs, double tol, int restart, int max_applies,
                    cudaStream_t st, double* info) {
  void *zo = slot(h, 0, nrhs), *wo = slot(h, 1, nrhs), *be = slot(h, 2, nrhs), *bo = slot(h, 3, nrhs);
  void *rhs = slot(h, 4, nrhs), *xe = slot(h, 5, nrhs);
  AMG_TRY_INTERNAL(split_merge(h, true, b, be, bo, nrhs, st));
  // reduced right-hand side b_e - D_eo D_oo^-1 b_o
  AMG_TRY_INTERNAL(amg_internal_eo_apply(h, 1, 0, 1, true, bo, false, nullptr, 0.0, false, nullptr, 0.0, wo, nullptr,
                                         nullptr, nullptr, nrhs, st));
  AMG_TRY_INTERNAL(amg_internal_eo_apply(h, 0, 1, 9, false, nullptr, false, wo, -1.0, false, be, 1.0, rhs, nullptr,
                                         nullptr, nullptr, nrhs, st));
  AMG_TRY_INTERNAL(amg_internal_solve_op(h, (h->g.Vc / 2) * h->g.nc, amg_internal_schur_apply, rhs, xe, nrhs, tol,
                                         restart, max_applies, st, info));
  // x_o = D_oo^-1 (b_o - D_oe x_e), one pass
  AMG_TRY_INTERNAL(amg_internal_eo_apply(h, 1, 1, 9, false, nullptr, false, xe, -1.0, false, bo, 1.0, wo, nullptr,
                                         nullptr, nullptr, nrhs, st, true));
  return split_merge(h, false, xe, wo, x, nrhs, st);
}

}  // namespace

amg_status amg_internal_schur_apply(amg_coarse* h, const void* xe, void* ye, int nrhs, cudaStream_t st,
                                    const int* skip, const double* xscale, void* vout) {
  void* wo = slot(h, 1, nrhs);
  const bool sc = xscale != nullptr;
  // w_o = D_oo^-1 D_oe x_e (hops and inverse in one pass), then y_e = D_ee x_e - D_eo w_o
  AMG_TRY_INTERNAL(amg_internal_eo_apply(h, 1, 1, 9, false, nullptr, false, xe, 1.0, sc, nullptr, 0.0, wo, nullptr,
                                         xscale, skip, nrhs, st, true));
  return amg_internal_eo_apply(h, 0, 0, 9, false, xe, sc, wo, -1.0, false, nullptr, 0.0, ye, vout, xscale, skip, nrhs,
                               st);
}

extern "C" amg_status amg_setup_evenodd(amg_handle h, void* stream) {
  if (!h) return AMG_ERR_INVALID_ARG;
  if (h->level != 1) return AMG_ERR_UNSUPPORTED;  // not offered on a level-2 handle
  const Geom& g = h->g;
  for (int mu = 0; mu < 4; ++mu)
    if (g.Lc[mu] % 2) return AMG_ERR_UNSUPPORTED;
  const bool fp64 = h->p.link_prec == AMG_FP64 && h->p.vec_prec == AMG_FP64;
  const bool fp32 = h->p.link_prec == AMG_FP32 && h->p.vec_prec == AMG_FP32;
  if (!fp64 && !fp32) return AMG_ERR_UNSUPPORTED;
  if (g.nc > 64) return AMG_ERR_UNSUPPORTED;
  if (eo_ready(h)) return AMG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  const long long Vh = g.Vc / 2;
  std::vector<int> site(2 * Vh);
  for (long long i = 0; i < g.Vc; ++i) {
    const long long x = i % g.Lc[0], y = (i / g.Lc[0]) % g.Lc[1], z = (i / ((long long)g.Lc[0] * g.Lc[1])) % g.Lc[2],
                    t = i / ((long long)g.Lc[0] * g.Lc[1] * g.Lc[2]);
    site[((x + y + z + t) & 1) * Vh + (i >> 1)] = (int)i;
  }
  const size_t n2 = (size_t)Vh * g.nc * g.nc;
  const int nrmax = h->p.max_nrhs < 16 ? h->p.max_nrhs : 16;
  auto fail = [&](amg_status s) {
    cudaFree(h->eo_site);
    cudaFree(h->Dinv64);
    cudaFree(h->Dinvq);
    cudaFree(h->eo_tmp);
    h->eo_site = nullptr;
    h->Dinv64 = nullptr;
    h->Dinvq = nullptr;
    h->eo_tmp = nullptr;
    return s;
  };
  if (cudaMalloc(&h->eo_site, site.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->Dinv64, n2 * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&h->Dinvq, n2 * (fp64 ? sizeof(double2) : sizeof(float2))) != cudaSuccess ||
      cudaMalloc(&h->eo_tmp, kSlots * half_bytes(h, nrmax)) != cudaSuccess) {
    amg_note_error("amg_setup_evenodd: device allocation failed");
    return fail(AMG_ERR_OOM);
  }
  h->eo_tmp_bytes = kSlots * half_bytes(h, nrmax);
  if (cudaMemcpyAsync(h->eo_site, site.data(), site.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(AMG_ERR_CUDA);
  const size_t smem = (2 * (size_t)g.nc * g.nc + g.nc) * sizeof(double2);
  if (cudaFuncSetAttribute(self_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return fail(AMG_ERR_CUDA);
  self_inverse_kernel<<<(unsigned)Vh, 256, smem, st>>>(h->Dc64, h->eo_site + Vh, g.nc, h->Dinv64, h->Dinvq, fp64,
                                                        h->err);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    amg_note_error("amg_setup_evenodd: self-block inverse failed");
    return fail(AMG_ERR_CUDA);
  }
  h->launches++;
  unsigned e = 0;
  cudaMemcpy(&e, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e & AMG_EBIT_NONFINITE) {
    cudaMemset(h->err, 0, sizeof(unsigned));
    return fail(AMG_ERR_NONFINITE);
  }
  return AMG_OK;
}

extern "C" amg_status amg_schur_apply(amg_handle h, const void* d_xe, void* d_ye, int nrhs, void* stream) {
  amg_status s = check_eo_vec(h, d_xe, d_ye, nrhs);
  if (s != AMG_OK) return s;
  h->last_stream = (cudaStream_t)stream;
  return amg_internal_schur_apply(h, d_xe, d_ye, nrhs, (cudaStream_t)stream, nullptr, nullptr, nullptr);
}

extern "C" amg_status amg_coarse_solve_eo(amg_handle h, const void* d_b, void* d_x, int nrhs, double tol, int restart,
                                          int max_applies, void* stream, double* info) {
  amg_status s = check_eo_vec(h, d_b, d_x, nrhs);
  if (s != AMG_OK) return s;
  if (!(tol >= 0) || restart < 1 || max_applies < 1) return AMG_ERR_INVALID_ARG;
  h->last_stream = (cudaStream_t)stream;
  return eo_solve(h, d_b, d_x, nrhs, tol, restart, max_applies, (cudaStream_t)stream, info);
}

extern "C" amg_status amg_cgc_eo(amg_handle h, const void* d_y, void* d_x, int nrhs, double tol, int restart,
                                 int max_applies, void* stream, double* info) {
  if (!h || !d_y || !d_x || !aligned16(d_y) || !aligned16(d_x)) return AMG_ERR_INVALID_ARG;
  if (nrhs < 1 || nrhs > 16 || nrhs > h->p.max_nrhs) return AMG_ERR_INVALID_ARG;
  if (!eo_ready(h)) return AMG_ERR_UNSUPPORTED;
  if (!(tol >= 0) || restart < 1 || max_applies < 1) return AMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  const size_t bytes = (size_t)h->g.Vc * h->g.nc * nrhs * coarse_elem_bytes(h);
  if (bytes > h->tmp_bytes) {
    cudaStreamSynchronize(st);
    cudaFree(h->xc_tmp);
    cudaFree(h->yc_tmp);
    h->xc_tmp = h->yc_tmp = nullptr;
    h->tmp_bytes = 0;
    if (cudaMalloc(&h->xc_tmp, bytes) != cudaSuccess || cudaMalloc(&h->yc_tmp, bytes) != cudaSuccess) {
      amg_note_error("amg_cgc_eo: device allocation failed");
      return AMG_ERR_OOM;
    }
    h->tmp_bytes = bytes;
  }
  AMG_TRY_INTERNAL(amg_internal_restrict(h, d_y, h->yc_tmp, nrhs, st));
  AMG_TRY_INTERNAL(eo_solve(h, h->yc_tmp, h->xc_tmp, nrhs, tol, restart, max_applies, st, info));
  return amg_internal_prolong(h, h->xc_tmp, d_x, nrhs, st);
}

extern "C" amg_status amg_export_Dinv(amg_handle h, void* out) {
  if (!h || !out) return AMG_ERR_INVALID_ARG;
  if (!h->Dinv64) return AMG_ERR_UNSUPPORTED;
  AMG_CUDA_TRY(cudaStreamSynchronize(h->last_stream));
  AMG_CUDA_TRY(cudaMemcpy(out, h->Dinv64, (size_t)(h->g.Vc / 2) * h->g.nc * h->g.nc * sizeof(double2),
                          cudaMemcpyDefault));
  return AMG_OK;
}
