// A third level: the coarse lattice coarsened once more, and the two-grid cycle on level 1 that
// takes the place of the coarse solve (Sec. 3 builds two levels; the method carries over to
// three save for a coarse-grid smoother, which the paper does not have: here minimal-residual
// steps on D_c).
//
// Level-2 aggregates are blocks B2 of coarse sites, one aggregate per chirality (the l and r
// halves of a coarse site's 2 ntv1 components); dof n of an aggregate is (site v in the block,
// lexicographic x fastest; component k), n = v ntv1 + k.  R2 = per-aggregate classical
// Gram-Schmidt of the level-2 test vectors (projections applied twice, as Alg. 5 on the fine
// grid), P2 = R2^dag, D_cc = R2 D_c P2 (Eq. cgo): the block of D_cc between aggregate i and its
// level-2 neighbour in direction d collects the couplings D_c[s][e] of sites s of i whose hop e
// leaves the block through the face d (d = 0: hops that stay inside).  Everything is FP64 in the
// setup; the level-2 handle then stores D_cc in its link precision like any coarse handle.
#include "amg_internal.cuh"

#include <new>
#include <vector>

namespace {

// Local coordinates in the level-2 block and the block (aggregate) of a level-1 site s (g: the
// level-2 geometry, g.L = the level-1 lattice).
__device__ inline void l2_locate(const Geom& g, long long s, int lc[4], long long& blk, int& v) {
  int c[4];
  long long r = s;
  for (int mu = 0; mu < 4; ++mu) {
    c[mu] = (int)(r % g.L[mu]);
    r /= g.L[mu];
  }
  int b[4];
  for (int mu = 0; mu < 4; ++mu) {
    b[mu] = c[mu] / g.B[mu];
    lc[mu] = c[mu] - b[mu] * g.B[mu];
  }
  blk = (((long long)b[3] * g.Lc[2] + b[2]) * g.Lc[1] + b[1]) * g.Lc[0] + b[0];
  v = ((lc[3] * g.B[2] + lc[2]) * g.B[1] + lc[1]) * g.B[0] + lc[0];
}

// CTA-wide complex sum (blockDim.x a multiple of 32, at most 1024); every thread gets the result.
__device__ inline double2 l2_block_sum(double2 v, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();  // sh may still be read by the previous call
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double2 t = make_double2(0, 0);
  for (int w = 0; w < nw; ++w) t = cadd(t, sh[w]);
  return t;
}

// R2 of aggregate blockIdx.x / 2, chirality blockIdx.x % 2: the test vectors tv2 ([Vc1][2][ntv1]
// [ntv2]) on the aggregate, classical Gram-Schmidt with the projections applied twice, in order
// j = 0 .. ntv2 - 1, in place in the rows of R (stored conj(q_j) at the end).  A vector whose
// norm falls below 1e-12 of its norm before the projections sets the rank bit.
__global__ void __launch_bounds__(256) gs2_kernel(const double2* __restrict__ tv2, double2* __restrict__ R, Geom g,
                                                  int ntv1, unsigned* err) {
  __shared__ double2 sh[32];
  __shared__ double2 cf[AMG_MAX_NTV];
  const long long i = blockIdx.x >> 1;
  const int h = blockIdx.x & 1;
  const int ntv2 = g.ntv, n = g.nagg;
  double2* Ri = R + (i * 2 + h) * (long long)ntv2 * n;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int v = e / ntv1, k = e - v * ntv1;
    const long long s = block_site(g, i, v);
    for (int j = 0; j < ntv2; ++j) Ri[(long long)j * n + e] = tv2[((s * 2 + h) * ntv1 + k) * ntv2 + j];
  }
  __syncthreads();
  for (int j = 0; j < ntv2; ++j) {
    double2* w = Ri + (long long)j * n;
    double2 p = make_double2(0, 0);
    for (int e = threadIdx.x; e < n; e += blockDim.x) p.x += w[e].x * w[e].x + w[e].y * w[e].y;
    const double wnorm = sqrt(l2_block_sum(p, sh).x);
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = 0; q < j; ++q) {  // every coefficient from the same w
        const double2* Rq = Ri + (long long)q * n;
        double2 c = make_double2(0, 0);
        for (int e = threadIdx.x; e < n; e += blockDim.x) cfmac(c, Rq[e], w[e]);
        c = l2_block_sum(c, sh);
        if (threadIdx.x == 0) cf[q] = c;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        double2 a = w[e];
        for (int q = 0; q < j; ++q) {
          const double2 b = Ri[(long long)q * n + e];
          const double2 c = cf[q];
          a.x -= c.x * b.x - c.y * b.y;
          a.y -= c.x * b.y + c.y * b.x;
        }
        w[e] = a;
      }
      __syncthreads();
    }
    p = make_double2(0, 0);
    for (int e = threadIdx.x; e < n; e += blockDim.x) p.x += w[e].x * w[e].x + w[e].y * w[e].y;
    const double nrm = sqrt(l2_block_sum(p, sh).x);
    if (!(nrm > 1e-12 * wnorm)) {
      if (threadIdx.x == 0) atomicOr(err, AMG_EBIT_RANK);
    }
    const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) w[e] = cscale(w[e], inv);
    __syncthreads();
  }
  for (long long e = threadIdx.x; e < (long long)ntv2 * n; e += blockDim.x) Ri[e] = cconj(Ri[e]);
}

// D_cc block (aggregate blockIdx.x, direction blockIdx.y), canonical [row][col]: entry (a, b),
// a = (h, j), b = (h', j'), = sum over sites s of the aggregate and hops e of class d of
// q_{i,h,j}(s)^dag D_c[s][e] q_{nbr,h',j'}(s + e), with q = conj(R row).
__global__ void __launch_bounds__(256) assemble2_kernel(const double2* __restrict__ Dc1, const int* __restrict__ nbr1,
                                                        const double2* __restrict__ R, double2* __restrict__ Dcc,
                                                        Geom g, int ntv1) {
  const long long i = blockIdx.x;
  const int d = blockIdx.y;
  const int ntv2 = g.ntv, nc2 = g.nc, n = g.nagg, nc1 = 2 * ntv1;
  for (int ab = threadIdx.x; ab < nc2 * nc2; ab += blockDim.x) {
    const int a = ab / nc2, b = ab - a * nc2;
    const int h = a / ntv2, j = a - h * ntv2, hp = b / ntv2, jp = b - hp * ntv2;
    const double2* Ra = R + ((i * 2 + h) * ntv2 + j) * (long long)n;
    double2 acc = make_double2(0, 0);
    for (int v = 0; v < (int)g.Vb; ++v) {
      const long long s = block_site(g, i, v);
      int lc[4];
      {
        int q = v;
        for (int mu = 0; mu < 4; ++mu) {
          lc[mu] = q % g.B[mu];
          q /= g.B[mu];
        }
      }
      for (int e = 0; e < 9; ++e) {
        int cls = 0;
        if (e > 0) {
          const int mu = (e - 1) >> 1;
          if (e & 1) cls = lc[mu] == g.B[mu] - 1 ? e : 0;
          else cls = lc[mu] == 0 ? e : 0;
        }
        if (cls != d) continue;
        const long long se = __ldg(nbr1 + s * 9 + e);
        int lce[4], ve;
        long long ie;
        l2_locate(g, se, lce, ie, ve);
        const double2* Rb = R + ((ie * 2 + hp) * ntv2 + jp) * (long long)n + (long long)ve * ntv1;
        const double2* D = Dc1 + (s * 9 + e) * (long long)nc1 * nc1;
        for (int k = 0; k < ntv1; ++k) {
          double2 t = make_double2(0, 0);  // sum_k' D[h k][h' k'] conj(Rb[k'])
          const double2* Drow = D + (long long)(h * ntv1 + k) * nc1 + hp * ntv1;
          for (int kp = 0; kp < ntv1; ++kp) cfma(t, Drow[kp], cconj(Rb[kp]));
          cfma(acc, Ra[(long long)v * ntv1 + k], t);
        }
      }
    }
    Dcc[((i * 9 + d) * nc2 + a) * (long long)nc2 + b] = acc;
  }
}

// Canonical FP64 D_cc -> the apply layout [Vc][9][nc col][nc row] in T2 (double2 or float2).
template <typename T2>
__global__ void dcc_store_kernel(const double2* __restrict__ Dc, T2* __restrict__ out, long long nblk, int nc) {
  const long long total = nblk * nc * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / ((long long)nc * nc);
    const int r = (int)(e - blk * nc * nc), col = r / nc, row = r - col * nc;
    const double2 v = Dc[blk * nc * nc + (long long)row * nc + col];
    T2 o;
    o.x = v.x;
    o.y = v.y;
    out[e] = o;
  }
}

template <typename C> __device__ inline double2 l2_d(C v) { return make_double2((double)v.x, (double)v.y); }
template <typename C> __device__ inline C l2_c(double2 v) {
  C o;
  o.x = v.x;
  o.y = v.y;
  return o;
}

// y_cc = R2 y_c: one thread per level-2 entry (aggregate, chirality, vector, column).
template <typename C>
__global__ void restrict2_kernel(const double2* __restrict__ R, const C* __restrict__ yc, C* __restrict__ ycc, Geom g,
                                 int ntv1, int nrhs) {
  const int ntv2 = g.ntv, n = g.nagg;
  const long long total = g.Vc * 2 * ntv2 * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % nrhs);
    const long long row = e / nrhs;  // (i, h, j)
    const long long ih = row / ntv2;
    const long long i = ih >> 1;
    const int h = (int)(ih & 1);
    const double2* Rr = R + row * n;
    double2 acc = make_double2(0, 0);
    for (int v = 0; v < (int)g.Vb; ++v) {
      const long long s = block_site(g, i, v);
      const C* y = yc + (s * 2 + h) * (long long)ntv1 * nrhs + r;
      for (int k = 0; k < ntv1; ++k) cfma(acc, Rr[(long long)v * ntv1 + k], l2_d(y[(long long)k * nrhs]));
    }
    ycc[e] = l2_c<C>(acc);
  }
}

// x_c = P2 x_cc (add: x_c += P2 x_cc): one thread per level-1 entry (site, chirality, component,
// column).
template <typename C>
__global__ void prolong2_kernel(const double2* __restrict__ R, const C* __restrict__ xcc, C* __restrict__ xc, Geom g,
                                int ntv1, int nrhs, int add) {
  const int ntv2 = g.ntv, n = g.nagg;
  const long long total = g.V * 2 * ntv1 * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % nrhs);
    long long q = e / nrhs;
    const int k = (int)(q % ntv1);
    q /= ntv1;
    const int h = (int)(q & 1);
    const long long s = q >> 1;
    int lc[4], v;
    long long i;
    l2_locate(g, s, lc, i, v);
    double2 acc = make_double2(0, 0);
    const double2* Rr = R + (i * 2 + h) * (long long)ntv2 * n + (long long)v * ntv1 + k;
    const C* x = xcc + (i * 2 + h) * (long long)ntv2 * nrhs + r;
    for (int j = 0; j < ntv2; ++j) cfmac(acc, Rr[(long long)j * n], l2_d(x[(long long)j * nrhs]));
    if (add) acc = cadd(acc, l2_d(xc[e]));
    xc[e] = l2_c<C>(acc);
  }
}

// w = y - w and x += e over n complex entries.
template <typename C>
__global__ void l2_sub_kernel(const C* __restrict__ y, C* __restrict__ w, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    C a = y[e];
    const C b = w[e];
    a.x -= b.x;
    a.y -= b.y;
    w[e] = a;
  }
}
template <typename C>
__global__ void l2_add_kernel(C* __restrict__ x, const C* __restrict__ v, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    C a = x[e];
    const C b = v[e];
    a.x += b.x;
    a.y += b.y;
    x[e] = a;
  }
}

amg_status l2_alloc(void** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA;
  }
  return AMG_OK;
}

void l2_free(amg_coarse* h) {
  cudaFree(h->R64);
  cudaFree(h->Dc64);
  cudaFree(h->Dq);
  cudaFree(h->nbr);
  cudaFree(h->err);
  delete h;
}

int l2_ntv1(const amg_coarse* h2) { return (int)(h2->g.nagg / h2->g.Vb); }

template <typename C>
amg_status restrict2_launch(amg_coarse* h2, const void* yc, void* ycc, int nrhs, cudaStream_t st) {
  restrict2_kernel<C><<<4 * amg_sm_count(), 128, 0, st>>>(h2->R64, (const C*)yc, (C*)ycc, h2->g, l2_ntv1(h2), nrhs);
  AMG_LAUNCH_CHECK();
  h2->launches++;
  return AMG_OK;
}
template <typename C>
amg_status prolong2_launch(amg_coarse* h2, const void* xcc, void* xc, int nrhs, bool add, cudaStream_t st) {
  prolong2_kernel<C><<<4 * amg_sm_count(), 128, 0, st>>>(h2->R64, (const C*)xcc, (C*)xc, h2->g, l2_ntv1(h2), nrhs,
                                                          add ? 1 : 0);
  AMG_LAUNCH_CHECK();
  h2->launches++;
  return AMG_OK;
}
amg_status restrict2_any(amg_coarse* h2, const void* yc, void* ycc, int nrhs, cudaStream_t st) {
  return h2->p.vec_prec == AMG_FP64 ? restrict2_launch<double2>(h2, yc, ycc, nrhs, st)
                                    : restrict2_launch<float2>(h2, yc, ycc, nrhs, st);
}
amg_status prolong2_any(amg_coarse* h2, const void* xcc, void* xc, int nrhs, bool add, cudaStream_t st) {
  return h2->p.vec_prec == AMG_FP64 ? prolong2_launch<double2>(h2, xcc, xc, nrhs, add, st)
                                    : prolong2_launch<float2>(h2, xcc, xc, nrhs, add, st);
}

template <typename C>
amg_status vec_op(bool sub, const void* a, void* b, long long n, cudaStream_t st) {
  if (sub) l2_sub_kernel<C><<<4 * amg_sm_count(), 256, 0, st>>>((const C*)a, (C*)b, n);
  else l2_add_kernel<C><<<4 * amg_sm_count(), 256, 0, st>>>((C*)b, (const C*)a, n);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// One two-grid cycle on level 1 (see amg_two_grid in amg.h).
amg_status two_grid_impl(amg_coarse* h1, const void* yc, void* xc, int nrhs, cudaStream_t st) {
  amg_coarse* h2 = h1->next;
  const amg_level2_params& lp = h1->l2p;
  const size_t eb = coarse_elem_bytes(h1);
  const long long n1 = h1->g.Vc * h1->g.nc * nrhs, n2 = h2->g.Vc * h2->g.nc * nrhs;
  const size_t b1 = ((size_t)n1 * eb + 255) / 256 * 256, b2 = ((size_t)n2 * eb + 255) / 256 * 256;
  const size_t need = 2 * b1 + 2 * b2;
  if (need > h1->l2work_bytes) {
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(h1->l2work);
    h1->l2work = nullptr;
    h1->l2work_bytes = 0;
    AMG_TRY_INTERNAL(l2_alloc(&h1->l2work, need));
    h1->l2work_bytes = need;
  }
  unsigned char* w = (unsigned char*)h1->l2work;
  void* r = w;
  void* e = w + b1;
  void* ycc = w + 2 * b1;
  void* xcc = w + 2 * b1 + b2;
  const bool f64 = h1->p.vec_prec == AMG_FP64;
  auto sub = [&](const void* a, void* b) { return f64 ? vec_op<double2>(true, a, b, n1, st) : vec_op<float2>(true, a, b, n1, st); };
  auto add = [&](const void* a, void* b) { return f64 ? vec_op<double2>(false, a, b, n1, st) : vec_op<float2>(false, a, b, n1, st); };
  const int mr_applies = 2 * lp.n_mr - 1;
  // pre-smoothing x = MR(y) from zero, residual r = y - D_c x
  if (lp.n_mr > 0) {
    AMG_TRY_INTERNAL(amg_internal_solve(h1, yc, xc, nrhs, 0.0, 1, mr_applies, st, nullptr));
    AMG_TRY_INTERNAL(amg_internal_apply(h1, xc, r, nrhs, st));
    AMG_TRY_INTERNAL(sub(yc, r));
  } else {
    AMG_CUDA_TRY(cudaMemsetAsync(xc, 0, (size_t)n1 * eb, st));
    AMG_CUDA_TRY(cudaMemcpyAsync(r, yc, (size_t)n1 * eb, cudaMemcpyDeviceToDevice, st));
  }
  // coarse correction x += P2 D_cc^{-1} R2 r
  AMG_TRY_INTERNAL(restrict2_any(h2, r, ycc, nrhs, st));
  AMG_TRY_INTERNAL(amg_internal_solve(h2, ycc, xcc, nrhs, lp.tol, lp.restart, lp.max_applies, st, nullptr));
  AMG_TRY_INTERNAL(prolong2_any(h2, xcc, xc, nrhs, true, st));
  // post-smoothing x += MR(y - D_c x)
  if (lp.n_mr > 0) {
    AMG_TRY_INTERNAL(amg_internal_apply(h1, xc, r, nrhs, st));
    AMG_TRY_INTERNAL(sub(yc, r));
    AMG_TRY_INTERNAL(amg_internal_solve(h1, r, e, nrhs, 0.0, 1, mr_applies, st, nullptr));
    AMG_TRY_INTERNAL(add(e, xc));
  }
  h1->launches += lp.n_mr > 0 ? 3 : 0;
  return AMG_OK;
}

amg_status l2_check_vec(amg_coarse* h, const void* a, const void* b, int nrhs) {
  if (!h || !a || !b || a == b || !aligned16(a) || !aligned16(b)) return AMG_ERR_INVALID_ARG;
  if (nrhs < 1 || nrhs > h->p.max_nrhs) return AMG_ERR_INVALID_ARG;
  return AMG_OK;
}

}  // namespace

amg_status amg_internal_cgc3(amg_coarse* h, const void* y, void* x, int nrhs, cudaStream_t st) {
  if (!h->next || nrhs > h->next->p.max_nrhs) return AMG_ERR_INVALID_ARG;
  const size_t bytes = (size_t)h->g.Vc * h->g.nc * nrhs * coarse_elem_bytes(h);
  if (bytes > h->tmp_bytes) {
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(h->xc_tmp);
    cudaFree(h->yc_tmp);
    h->xc_tmp = h->yc_tmp = nullptr;
    h->tmp_bytes = 0;
    AMG_TRY_INTERNAL(l2_alloc(&h->xc_tmp, bytes));
    AMG_TRY_INTERNAL(l2_alloc(&h->yc_tmp, bytes));
    h->tmp_bytes = bytes;
  }
  AMG_TRY_INTERNAL(amg_internal_restrict(h, y, h->yc_tmp, nrhs, st));
  AMG_TRY_INTERNAL(two_grid_impl(h, h->yc_tmp, h->xc_tmp, nrhs, st));
  return amg_internal_prolong(h, h->xc_tmp, x, nrhs, st);
}

extern "C" {

amg_status amg_setup_level2(amg_handle h1, const amg_params* p2, const void* d_tv2, void* stream, amg_handle* out) {
  if (!out) return AMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!h1 || !p2 || !d_tv2 || !aligned16(d_tv2) || h1->level != 1) return AMG_ERR_INVALID_ARG;
  long long Vb2 = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (p2->L[mu] != h1->g.Lc[mu] || p2->B[mu] < 1 || p2->L[mu] % p2->B[mu] || p2->L[mu] / p2->B[mu] < 2)
      return AMG_ERR_INVALID_ARG;
    Vb2 *= p2->B[mu];
  }
  const int ntv1 = h1->g.ntv;
  if (p2->ntv < 1 || p2->ntv > 32 || p2->ntv > ntv1 * Vb2) return AMG_ERR_INVALID_ARG;
  if (p2->max_nrhs < 1 || p2->max_nrhs > 64) return AMG_ERR_INVALID_ARG;
  if (p2->vec_prec != h1->p.vec_prec) return AMG_ERR_INVALID_ARG;
  if (p2->vec_prec != AMG_FP64 && p2->vec_prec != AMG_FP32) return AMG_ERR_UNSUPPORTED;
  if (p2->link_prec != p2->vec_prec || p2->r_prec != p2->vec_prec) return AMG_ERR_UNSUPPORTED;
  amg_coarse* h = new (std::nothrow) amg_coarse();
  if (!h) return AMG_ERR_OOM;
  h->p = *p2;
  h->level = 2;
  Geom& g = h->g;
  g.V = Vb2 = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.L[mu] = p2->L[mu];
    g.B[mu] = p2->B[mu];
    g.Lc[mu] = p2->L[mu] / p2->B[mu];
    g.V *= p2->L[mu];
    Vb2 *= p2->B[mu];
  }
  g.Vb = Vb2;
  g.Vc = g.V / g.Vb;
  g.ntv = p2->ntv;
  g.nc = 2 * p2->ntv;
  g.nagg = (int)(Vb2 * ntv1);
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  const size_t nR = (size_t)g.Vc * 2 * g.ntv * g.nagg, nD = (size_t)g.Vc * 9 * g.nc * g.nc;
  amg_status s = AMG_OK;
  if (s == AMG_OK) s = l2_alloc((void**)&h->R64, nR * sizeof(double2));
  if (s == AMG_OK) s = l2_alloc((void**)&h->Dc64, nD * sizeof(double2));
  if (s == AMG_OK) s = l2_alloc(&h->Dq, nD * (p2->link_prec == AMG_FP64 ? sizeof(double2) : sizeof(float2)));
  if (s == AMG_OK) s = l2_alloc((void**)&h->nbr, (size_t)g.Vc * 9 * sizeof(int));
  if (s == AMG_OK) s = l2_alloc((void**)&h->err, sizeof(unsigned));
  if (s != AMG_OK) {
    l2_free(h);
    return s;
  }
  h->Rq = h->R64;
  std::vector<int> nb((size_t)g.Vc * 9);
  for (long long i = 0; i < g.Vc; ++i) {
    int X[4];
    long long r = i;
    for (int mu = 0; mu < 4; ++mu) {
      X[mu] = (int)(r % g.Lc[mu]);
      r /= g.Lc[mu];
    }
    for (int d = 0; d < 9; ++d) {
      int Y[4] = {X[0], X[1], X[2], X[3]};
      if (d > 0) {
        const int mu = (d - 1) / 2;
        Y[mu] = (Y[mu] + ((d & 1) ? 1 : -1) + g.Lc[mu]) % g.Lc[mu];
      }
      nb[i * 9 + d] = (int)(((long long)(Y[3] * g.Lc[2] + Y[2]) * g.Lc[1] + Y[1]) * g.Lc[0] + Y[0]);
    }
  }
  auto fail = [&](amg_status e) {
    cudaStreamSynchronize(st);
    l2_free(h);
    return e;
  };
  if (cudaMemcpyAsync(h->nbr, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(h->err, 0, sizeof(unsigned), st) != cudaSuccess)
    return fail(AMG_ERR_CUDA);
  gs2_kernel<<<(unsigned)(g.Vc * 2), 128, 0, st>>>((const double2*)d_tv2, h->R64, g, ntv1, h->err);
  if (cudaGetLastError() != cudaSuccess) return fail(AMG_ERR_CUDA);
  assemble2_kernel<<<dim3((unsigned)g.Vc, 9), 256, 0, st>>>(h1->Dc64, h1->nbr, h->R64, h->Dc64, g, ntv1);
  if (cudaGetLastError() != cudaSuccess) return fail(AMG_ERR_CUDA);
  if (p2->link_prec == AMG_FP64)
    dcc_store_kernel<double2><<<4 * amg_sm_count(), 256, 0, st>>>(h->Dc64, (double2*)h->Dq, g.Vc * 9, g.nc);
  else
    dcc_store_kernel<float2><<<4 * amg_sm_count(), 256, 0, st>>>(h->Dc64, (float2*)h->Dq, g.Vc * 9, g.nc);
  if (cudaGetLastError() != cudaSuccess) return fail(AMG_ERR_CUDA);
  h->launches += 3;
  unsigned e = 0;
  if (cudaMemcpyAsync(&e, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(AMG_ERR_CUDA);
  if (e & ~AMG_EBIT_RANK) return fail(AMG_ERR_CUDA);
  if (e) {
    if (cudaMemsetAsync(h->err, 0, sizeof(unsigned), st) != cudaSuccess) return fail(AMG_ERR_CUDA);
    *out = h;
    return AMG_ERR_RANK_DEFICIENT;
  }
  *out = h;
  return AMG_OK;
}

amg_status amg_restrict2(amg_handle h2, const void* d_yc, void* d_ycc, int nrhs, void* stream) {
  AMG_TRY_INTERNAL(l2_check_vec(h2, d_yc, d_ycc, nrhs));
  if (h2->level != 2) return AMG_ERR_INVALID_ARG;
  h2->last_stream = (cudaStream_t)stream;
  return restrict2_any(h2, d_yc, d_ycc, nrhs, (cudaStream_t)stream);
}

amg_status amg_prolong2(amg_handle h2, const void* d_xcc, void* d_xc, int nrhs, void* stream) {
  AMG_TRY_INTERNAL(l2_check_vec(h2, d_xcc, d_xc, nrhs));
  if (h2->level != 2) return AMG_ERR_INVALID_ARG;
  h2->last_stream = (cudaStream_t)stream;
  return prolong2_any(h2, d_xcc, d_xc, nrhs, false, (cudaStream_t)stream);
}

amg_status amg_attach_level2(amg_handle h1, amg_handle h2, const amg_level2_params* lp) {
  if (!h1 || h1->level != 1) return AMG_ERR_INVALID_ARG;
  if (!h2) {
    if (h1->next) h1->next->prev = nullptr;
    h1->next = nullptr;
    return AMG_OK;
  }
  if (!lp || h2->level != 2 || lp->n_mr < 0 || lp->n_mr > 1000 || lp->restart < 1 || lp->restart > AMG_MAX_NTV ||
      lp->max_applies < 1 || !(lp->tol >= 0))
    return AMG_ERR_INVALID_ARG;
  for (int mu = 0; mu < 4; ++mu)
    if (h2->g.L[mu] != h1->g.Lc[mu]) return AMG_ERR_INVALID_ARG;
  if (h2->g.nagg != h2->g.Vb * h1->g.ntv || h2->p.vec_prec != h1->p.vec_prec) return AMG_ERR_INVALID_ARG;
  if (h2->prev && h2->prev != h1) h2->prev->next = nullptr;
  if (h1->next && h1->next != h2) h1->next->prev = nullptr;
  h1->next = h2;
  h2->prev = h1;
  h1->l2p = *lp;
  return AMG_OK;
}

amg_status amg_two_grid(amg_handle h1, const void* d_yc, void* d_xc, int nrhs, void* stream) {
  AMG_TRY_INTERNAL(l2_check_vec(h1, d_yc, d_xc, nrhs));
  if (h1->level != 1 || !h1->next || nrhs > h1->next->p.max_nrhs) return AMG_ERR_INVALID_ARG;
  h1->last_stream = (cudaStream_t)stream;
  return two_grid_impl(h1, d_yc, d_xc, nrhs, (cudaStream_t)stream);
}

}  // extern "C"
