// Restriction y_c = R y (Eq. R, Alg. 6), coarse-operator application y_c = D_c x_c (Alg. 2) and
// prolongation x = P x_c, P = R^dagger (Alg. 2), as streaming SIMT kernels for FP64 / FP32 /
// FP16-scaled storage and a few right-hand sides.
//
// All three are HBM-bound streams of R or D_c that are read exactly once per call.  Each CTA
// owns one block (R, P) or one coarse site (D_c) and reads its matrix as one contiguous run of
// 16-byte loads; the small vector it multiplies is staged in shared memory first.
#include "amg_internal.cuh"

namespace {

template <typename T> struct Acc;
template <> struct Acc<double2> { using type = double2; };
template <> struct Acc<float2> { using type = float2; };
template <> struct Acc<__half2> { using type = float2; };

// Complex values per 16-byte load.
template <typename T> struct Pack;
template <> struct Pack<double2> {
  static constexpr int CPL = 1;
  __device__ static void load(const double2* p, double2 (&v)[1]) { v[0] = __ldg(p); }
};
template <> struct Pack<float2> {
  static constexpr int CPL = 2;
  __device__ static void load(const float2* p, float2 (&v)[2]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = make_float2(t.x, t.y);
    v[1] = make_float2(t.z, t.w);
  }
};
template <> struct Pack<__half2> {
  static constexpr int CPL = 4;
  __device__ static void load(const __half2* p, float2 (&v)[4]) {
    const uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
    const unsigned u[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __half2 hv;
      memcpy(&hv, &u[k], 4);
      v[k] = __half22float2(hv);
    }
  }
};

template <typename T>
__device__ inline T warp_csum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// ---------------------------------------------------------------- restriction
// One CTA per block.  y on the block is staged as [h][n][r]; warp w computes rows (h, j) of
// R_i^h y_i^h, the lanes striding over n with 16-byte loads of the row, then a shuffle sum.
template <typename ST, int NR>
__global__ void __launch_bounds__(256) restrict_kernel(const ST* __restrict__ R, const ST* __restrict__ y,
                                                       ST* __restrict__ yc, Geom g, int ld, int r0) {
  using AT = typename Acc<ST>::type;
  constexpr int CPL = Pack<ST>::CPL;
  extern __shared__ __align__(16) unsigned char smraw[];
  AT* ys = reinterpret_cast<AT*>(smraw);
  const long long blk = blockIdx.x;
  const int nagg = g.nagg, ntv = g.ntv, Vb = (int)g.Vb;
  for (int e = threadIdx.x; e < Vb * 12 * NR; e += blockDim.x) {
    const int sl = e / (12 * NR), rem = e % (12 * NR), dof = rem / NR, r = rem % NR;
    const long long site = block_site(g, blk, sl);
    const int hh = dof / 6, n = sl * 6 + dof % 6;
    ys[((size_t)hh * nagg + n) * NR + r] = y[(site * 12 + dof) * ld + r0 + r];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int row = warp; row < 2 * ntv; row += nw) {
    const int hh = row / ntv, j = row % ntv;
    const ST* Rrow = R + ((blk * 2 + hh) * ntv + j) * (long long)nagg;
    const AT* yh = ys + (size_t)hh * nagg * NR;
    AT acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = AT{0, 0};
#pragma unroll 4
    for (int q = lane; q < nagg / CPL; q += 32) {
      ST v[CPL];
      Pack<ST>::load(Rrow + q * CPL, v);
#pragma unroll
      for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int r = 0; r < NR; ++r) cfma(acc[r], v[k], yh[(q * CPL + k) * NR + r]);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const AT s = warp_csum(acc[r]);
      if (lane == 0) yc[((blk * 2 + hh) * ntv + j) * ld + r0 + r] = s;
    }
  }
}

// ---------------------------------------------------------------- prolongation
// One CTA per block.  x_c of the block is staged in shared memory; a thread owns CPL consecutive
// fine dofs of one site (one chirality) and sums conj(R[h][j][n]) x_c[h][j] over j, reading R
// coalesced across the threads.
template <typename ST, int NR>
__global__ void __launch_bounds__(256) prolong_kernel(const ST* __restrict__ R, const ST* __restrict__ xc,
                                                      ST* __restrict__ x, Geom g, int ld, int r0) {
  using AT = typename Acc<ST>::type;
  constexpr int CPL = Pack<ST>::CPL;
  constexpr int TPS = 12 / CPL;  // tasks per site
  __shared__ AT xs[2 * AMG_MAX_NTV * NR];
  const long long blk = blockIdx.x;
  const int nagg = g.nagg, ntv = g.ntv, Vb = (int)g.Vb;
  for (int e = threadIdx.x; e < 2 * ntv * NR; e += blockDim.x)
    xs[e] = xc[(blk * 2 * ntv + e / NR) * ld + r0 + e % NR];
  __syncthreads();
  for (int t = threadIdx.x; t < Vb * TPS; t += blockDim.x) {
    const int sl = t / TPS, p = t % TPS, dof0 = p * CPL, hh = dof0 / 6;
    const int n0 = sl * 6 + dof0 % 6;
    const ST* Rp = R + (blk * 2 + hh) * (long long)ntv * nagg + n0;
    const AT* xh = xs + hh * ntv * NR;
    AT acc[CPL][NR];
#pragma unroll
    for (int k = 0; k < CPL; ++k)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[k][r] = AT{0, 0};
#pragma unroll 4
    for (int j = 0; j < ntv; ++j) {
      ST v[CPL];
      Pack<ST>::load(Rp + (long long)j * nagg, v);
#pragma unroll
      for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int r = 0; r < NR; ++r) cfmac(acc[k][r], v[k], xh[j * NR + r]);
    }
    const long long site = block_site(g, blk, sl);
    ST* xo = x + (site * 12 + dof0) * ld + r0;
    if (NR == 1 && CPL == 2 && ld == 1) {
      *reinterpret_cast<float4*>(xo) =
          make_float4((float)acc[0][0].x, (float)acc[0][0].y, (float)acc[CPL - 1][0].x, (float)acc[CPL - 1][0].y);
    } else {
#pragma unroll
      for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int r = 0; r < NR; ++r) xo[k * ld + r] = acc[k][r];
    }
  }
}

// ---------------------------------------------------------------- coarse operator
// One CTA per coarse site i.  The 9 neighbour vectors, each pre-multiplied by its block's scale,
// are staged as X[k = d*nc + b]; the site's links are stored column-major (At[d][b][a]) so the CTA
// streams them as one contiguous run: thread t keeps the rows rc*CPL.. of its 16-byte chunk fixed
// and walks the columns k = grp, grp + G, ...; the G partial row vectors are summed at the end.
template <typename LT, int NR>
__global__ void __launch_bounds__(512) apply_kernel(const LT* __restrict__ Dq, const float* __restrict__ scale,
                                                    const int* __restrict__ nbr,
                                                    const typename Acc<LT>::type* __restrict__ xc,
                                                    typename Acc<LT>::type* __restrict__ yc, Geom g, int ld,
                                                    int r0, int G, const int* __restrict__ skip) {
  using AT = typename Acc<LT>::type;
  using RT = decltype(AT{}.x);
  constexpr int CPL = Pack<LT>::CPL;
  extern __shared__ __align__(16) unsigned char smraw[];
  if (skip && *skip) return;
  const int nc = g.nc, K = 9 * nc, Gc = nc / CPL;
  AT* xs = reinterpret_cast<AT*>(smraw);       // [K][NR]
  AT* red = xs + (size_t)K * NR;               // [G][nc][NR]
  const long long i = blockIdx.x;
  for (int e = threadIdx.x; e < K * NR; e += blockDim.x) {
    const int k = e / NR, r = e % NR, d = k / nc, b = k % nc;
    const long long j = nbr[i * 9 + d];
    AT v = xc[(j * nc + b) * ld + r0 + r];
    if (scale) {
      const RT s = (RT)scale[i * 9 + d];
      v.x *= s;
      v.y *= s;
    }
    xs[e] = v;
  }
  __syncthreads();
  const int t = threadIdx.x, rc = t % Gc, grp = t / Gc;
  AT acc[CPL][NR];
#pragma unroll
  for (int q = 0; q < CPL; ++q)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[q][r] = AT{0, 0};
  if (grp < G) {
    const LT* base = Dq + i * (long long)K * nc + rc * CPL;
#pragma unroll 4
    for (int k = grp; k < K; k += G) {
      AT v[CPL];
      Pack<LT>::load(base + (long long)k * nc, v);
#pragma unroll
      for (int q = 0; q < CPL; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) cfma(acc[q][r], v[q], xs[k * NR + r]);
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q)
#pragma unroll
      for (int r = 0; r < NR; ++r) red[((size_t)grp * nc + rc * CPL + q) * NR + r] = acc[q][r];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nc * NR; e += blockDim.x) {
    AT s = AT{0, 0};
    for (int gg = 0; gg < G; ++gg) {
      const AT v = red[(size_t)gg * nc * NR + e];
      s.x += v.x;
      s.y += v.y;
    }
    yc[(i * nc + e / NR) * ld + r0 + e % NR] = s;
  }
}

constexpr int kMaxSmem = 227 * 1024;

template <typename ST, int NR>
amg_status launch_restrict(amg_coarse* h, const ST* R, const ST* y, ST* yc, int ld, int r0, cudaStream_t s) {
  using AT = typename Acc<ST>::type;
  const size_t sm = (size_t)2 * h->g.nagg * NR * sizeof(AT);
  if (sm > (size_t)kMaxSmem) return AMG_ERR_UNSUPPORTED;
  if (sm > 48 * 1024)
    AMG_CUDA_TRY(cudaFuncSetAttribute(restrict_kernel<ST, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  restrict_kernel<ST, NR><<<(unsigned)h->g.Vc, 256, sm, s>>>(R, y, yc, h->g, ld, r0);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

template <typename ST, int NR>
amg_status launch_prolong(amg_coarse* h, const ST* R, const ST* xc, ST* x, int ld, int r0, cudaStream_t s) {
  prolong_kernel<ST, NR><<<(unsigned)h->g.Vc, 256, 0, s>>>(R, xc, x, h->g, ld, r0);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

template <typename LT, int NR>
amg_status launch_apply(amg_coarse* h, const LT* D, const float* scale, const void* xc, void* yc, int ld, int r0,
                        cudaStream_t s, const int* skip) {
  using AT = typename Acc<LT>::type;
  constexpr int CPL = Pack<LT>::CPL;
  const int nc = h->g.nc;
  if (nc % CPL) return AMG_ERR_UNSUPPORTED;
  const int Gc = nc / CPL;
  int G = 256 / Gc;
  if (G < 1) G = 1;
  if (G > 9 * nc) G = 9 * nc;
  const int T = ((Gc * G + 31) / 32) * 32;
  const size_t sm = ((size_t)9 * nc * NR + (size_t)G * nc * NR) * sizeof(AT);
  if (sm > (size_t)kMaxSmem || T > 512) return AMG_ERR_UNSUPPORTED;
  if (sm > 48 * 1024)
    AMG_CUDA_TRY(cudaFuncSetAttribute(apply_kernel<LT, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  apply_kernel<LT, NR><<<(unsigned)h->g.Vc, T, sm, s>>>(D, scale, h->nbr, (const AT*)xc, (AT*)yc, h->g, ld, r0, G, skip);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

// Splits nrhs into chunks of 4, 2 and 1 right-hand sides.
template <typename F>
amg_status for_rhs_chunks(int nrhs, F&& f) {
  int r0 = 0;
  while (r0 < nrhs) {
    const int left = nrhs - r0;
    const int nr = left >= 4 ? 4 : (left >= 2 ? 2 : 1);
    amg_status st = f(r0, nr);
    if (st != AMG_OK) return st;
    r0 += nr;
  }
  return AMG_OK;
}

}  // namespace

amg_status amg_internal_restrict(amg_coarse* h, const void* y, void* yc, int nrhs, cudaStream_t s) {
  if (h->p.vec_prec == AMG_FP64) {
    const double2* R = h->R64;
    return for_rhs_chunks(nrhs, [&](int r0, int nr) {
      if (nr == 4) return launch_restrict<double2, 4>(h, R, (const double2*)y, (double2*)yc, nrhs, r0, s);
      if (nr == 2) return launch_restrict<double2, 2>(h, R, (const double2*)y, (double2*)yc, nrhs, r0, s);
      return launch_restrict<double2, 1>(h, R, (const double2*)y, (double2*)yc, nrhs, r0, s);
    });
  }
  if (h->p.vec_prec == AMG_FP32 && h->p.r_prec == AMG_FP32) {
    const float2* R = (const float2*)h->Rq;
    return for_rhs_chunks(nrhs, [&](int r0, int nr) {
      if (nr == 4) return launch_restrict<float2, 4>(h, R, (const float2*)y, (float2*)yc, nrhs, r0, s);
      if (nr == 2) return launch_restrict<float2, 2>(h, R, (const float2*)y, (float2*)yc, nrhs, r0, s);
      return launch_restrict<float2, 1>(h, R, (const float2*)y, (float2*)yc, nrhs, r0, s);
    });
  }
  return AMG_ERR_UNSUPPORTED;
}

amg_status amg_internal_prolong(amg_coarse* h, const void* xc, void* x, int nrhs, cudaStream_t s) {
  if (h->p.vec_prec == AMG_FP64) {
    const double2* R = h->R64;
    return for_rhs_chunks(nrhs, [&](int r0, int nr) {
      if (nr == 4) return launch_prolong<double2, 4>(h, R, (const double2*)xc, (double2*)x, nrhs, r0, s);
      if (nr == 2) return launch_prolong<double2, 2>(h, R, (const double2*)xc, (double2*)x, nrhs, r0, s);
      return launch_prolong<double2, 1>(h, R, (const double2*)xc, (double2*)x, nrhs, r0, s);
    });
  }
  if (h->p.vec_prec == AMG_FP32 && h->p.r_prec == AMG_FP32) {
    const float2* R = (const float2*)h->Rq;
    return for_rhs_chunks(nrhs, [&](int r0, int nr) {
      if (nr == 4) return launch_prolong<float2, 4>(h, R, (const float2*)xc, (float2*)x, nrhs, r0, s);
      if (nr == 2) return launch_prolong<float2, 2>(h, R, (const float2*)xc, (float2*)x, nrhs, r0, s);
      return launch_prolong<float2, 1>(h, R, (const float2*)xc, (float2*)x, nrhs, r0, s);
    });
  }
  return AMG_ERR_UNSUPPORTED;
}

amg_status amg_internal_apply(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s) {
  return amg_internal_apply_ex(h, xc, yc, nrhs, s, nullptr);
}

amg_status amg_internal_apply_ex(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s,
                                 const int* skip) {
  switch (h->p.link_prec) {
    case AMG_FP64:
      if (h->p.vec_prec != AMG_FP64) return AMG_ERR_UNSUPPORTED;
      return for_rhs_chunks(nrhs, [&](int r0, int nr) {
        const double2* D = (const double2*)h->Dq;
        if (nr == 4) return launch_apply<double2, 4>(h, D, nullptr, xc, yc, nrhs, r0, s, skip);
        if (nr == 2) return launch_apply<double2, 2>(h, D, nullptr, xc, yc, nrhs, r0, s, skip);
        return launch_apply<double2, 1>(h, D, nullptr, xc, yc, nrhs, r0, s, skip);
      });
    case AMG_FP32:
      if (h->p.vec_prec == AMG_FP64) return AMG_ERR_UNSUPPORTED;
      return for_rhs_chunks(nrhs, [&](int r0, int nr) {
        const float2* D = (const float2*)h->Dq;
        if (nr == 4) return launch_apply<float2, 4>(h, D, nullptr, xc, yc, nrhs, r0, s, skip);
        if (nr == 2) return launch_apply<float2, 2>(h, D, nullptr, xc, yc, nrhs, r0, s, skip);
        return launch_apply<float2, 1>(h, D, nullptr, xc, yc, nrhs, r0, s, skip);
      });
    case AMG_FP16_SCALED:
      if (h->p.vec_prec == AMG_FP64) return AMG_ERR_UNSUPPORTED;
      return for_rhs_chunks(nrhs, [&](int r0, int nr) {
        const __half2* D = (const __half2*)h->Dq;
        if (nr == 4) return launch_apply<__half2, 4>(h, D, h->Dscale, xc, yc, nrhs, r0, s, skip);
        if (nr == 2) return launch_apply<__half2, 2>(h, D, h->Dscale, xc, yc, nrhs, r0, s, skip);
        return launch_apply<__half2, 1>(h, D, h->Dscale, xc, yc, nrhs, r0, s, skip);
      });
    default:
      return AMG_ERR_UNSUPPORTED;
  }
}
