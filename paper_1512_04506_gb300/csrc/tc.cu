// Multi-right-hand-side forms of Alg. 2 on the tensor cores for nrhs = 4, 8, 12 or 16
// right-hand sides (FP32 accumulation):
//   coarse apply   y_c = D_c x_c   (D_c in BF16 Re/Im planes; Sec. 3 stores D_c in half precision)
//   restriction    y_c = R y       (R in BF16 Re/Im planes, y BF16)
//   prolongation   x   = R^dag x_c (x BF16)
// The kernels here run the bodies of tc_body.cuh over a grid-stride range of blocks or coarse
// sites with one bulk-copy ring per CTA; this file also holds the BF16 storage conversions.
#include "tc_body.cuh"

namespace {
using namespace amgtc;

// Coarse vector (FP32 [Vc][nc][nrhs], optionally times xscale[r]; the (scaled) FP32 vector is also
// stored to vout when given) -> BF16 rows [Vc][nc][xunits * 8], round to nearest even.
template <int NRHS>
__global__ void xc_to_bf16_kernel(const float2* __restrict__ x, __nv_bfloat162* __restrict__ X, long long rows,
                                  const double* __restrict__ xscale, float2* __restrict__ vout,
                                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int pitch = 4 * (NRHS / 4 + ((NRHS / 4) & 1 ? 0 : 1));  // (Re, Im) pairs per row
  const long long total = rows * NRHS;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % NRHS);
    float2 v = x[e];
    if (xscale) {
      const float f = (float)xscale[r];
      v.x *= f;
      v.y *= f;
    }
    if (vout) vout[e] = v;
    X[(e / NRHS) * pitch + r] = __floats2bfloat162_rn(v.x, v.y);
  }
}

template <int NRHS>
__global__ void __launch_bounds__(160, 1) apply_tc_kernel(const TcApplyArgs a, const int* skip, int ns) {
  if (skip && *skip) return;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  ring_init(pp, ns, (int)(blockDim.x >> 5) - 1);
  __syncthreads();
  const Ring rg{pp, sm + kPipeBytes, ns, tc_apply_chunk(a.g.nc, NRHS)};
  RingPos rp;
  apply_tc_items<NRHS>(a, rg, blockIdx.x, a.g.Vc, gridDim.x, rp);
  if (threadIdx.x == 0) drain(pp, rp.c, ns);
}

template <int NRHS>
__global__ void __launch_bounds__(160, 1) restrict_tc_kernel(const TcRPArgs a, int ns) {
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  ring_init(pp, ns, (int)(blockDim.x >> 5) - 1);
  __syncthreads();
  const Ring rg{pp, sm + kPipeBytes, ns, tc_restrict_chunk(a.g.ntv, NRHS)};
  RingPos rp;
  restrict_tc_items<NRHS>(a, rg, blockIdx.x, a.g.Vc, gridDim.x, rp);
  if (threadIdx.x == 0) drain(pp, rp.c, ns);
}

template <int NRHS>
__global__ void __launch_bounds__(160, 4) prolong_tc_kernel(const TcRPArgs a, int ns) {
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  ring_init(pp, ns, (int)(blockDim.x >> 5) - 1);
  __syncthreads();
  const Ring rg{pp, sm + kPipeBytes, ns, tc_prolong_chunk(a.g.ntv)};
  RingPos rp;
  prolong_tc_items<NRHS>(a, rg, blockIdx.x, a.g.Vc, gridDim.x, rp);
  if (threadIdx.x == 0) drain(pp, rp.c, ns);
}

template <int NRHS, bool RESTRICT>
amg_status launch_rp_tc(amg_coarse* h, const void* in, void* out, cudaStream_t st) {
  const Geom& g = h->g;
  const int threads = 32 + 64 * ((NRHS + 7) / 8);
  const size_t chunk = RESTRICT ? tc_restrict_chunk(g.ntv, NRHS) : tc_prolong_chunk(g.ntv);
  // the prolongation: 4 stages and a register cap for 4 CTAs per SM (measured best)
  int ns = RESTRICT ? (int)((60 * 1024) / chunk) : 4;
  ns = ns < 2 ? 2 : (ns > 8 ? 8 : ns);
  const size_t smem = kPipeBytes + ns * chunk;
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  auto kern = RESTRICT ? restrict_tc_kernel<NRHS> : prolong_tc_kernel<NRHS>;
  AMG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  if (per_sm < 1) return AMG_ERR_UNSUPPORTED;
  const long long gmax = (long long)per_sm * amg_sm_count();
  const int grid = capped_grid(h, g.Vc, gmax);
  TcRPArgs a{(const bf16*)h->Rtc, in, out, nullptr, true, h->err, g};
  kern<<<grid, threads, smem, st>>>(a, ns);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

// R64 [blk][h][j][n] (complex double) -> Rtc (BF16, round to nearest even)
__global__ void r_to_tc_kernel(const double2* __restrict__ R, bf16* __restrict__ out, Geom g) {
  const int ntv = g.ntv, nagg = g.nagg, cpb = (int)(g.Vb / 8);
  const long long total = g.Vc * 2LL * ntv * nagg;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e % nagg);
    const long long q = e / nagg;
    const int j = (int)(q % ntv), h = (int)((q / ntv) % 2);
    const long long blk = q / (2LL * ntv);
    const int site = n / 6, dp = n % 6, c = site / 8, sl = site % 8;
    const int off = tc_pos(j, dp, 6) * 8 + sl;
    const double2 v = R[e];
    const long long base = ((blk * cpb + c) * 2 + h) * 2;
    out[((base + 0) * ntv + j) * 48 + off] = __double2bfloat16(v.x);
    out[((base + 1) * ntv + j) * 48 + off] = __double2bfloat16(v.y);
  }
}

// D_c (canonical FP64 [Vc][9][nc][nc]) -> BF16 planes [Vc][9][2][nc][nc] with rotated row pieces,
// round to nearest even; bf16_to_dc_kernel is the inverse (for export).
__global__ void dc_to_bf16_kernel(const double2* __restrict__ Dc, bf16* __restrict__ out, int nc, long long nblk) {
  const long long n2 = (long long)nc * nc, total = nblk * n2;
  const int P = nc / 8;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / n2;
    const int rem = (int)(e % n2), row = rem / nc, col = rem % nc;
    const int off = row * nc + tc_pos(row, col / 8, P) * 8 + col % 8;
    const double2 v = Dc[e];
    out[blk * 2 * n2 + off] = __double2bfloat16(v.x);
    out[blk * 2 * n2 + n2 + off] = __double2bfloat16(v.y);
  }
}

__global__ void bf16_to_dc_kernel(const bf16* __restrict__ in, double2* __restrict__ out, int nc, long long nblk) {
  const long long n2 = (long long)nc * nc, total = nblk * n2;
  const int P = nc / 8;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / n2;
    const int rem = (int)(e % n2), row = rem / nc, col = rem % nc;
    const int off = row * nc + tc_pos(row, col / 8, P) * 8 + col % 8;
    out[e] = make_double2((double)__bfloat162float(in[blk * 2 * n2 + off]),
                          (double)__bfloat162float(in[blk * 2 * n2 + n2 + off]));
  }
}

// D_c (canonical FP64) -> FP32 planes [Vc][9][2][nc][nc], rows of 16-byte pieces (4 floats)
// rotated by tc_rot(row, nc / 4), round to nearest (the same FP32 values as the SIMT copy).
__global__ void dc_to_tf32_kernel(const double2* __restrict__ Dc, float* __restrict__ out, int nc, long long nblk) {
  const long long n2 = (long long)nc * nc, total = nblk * n2;
  const int P = nc / 4;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / n2;
    const int rem = (int)(e % n2), row = rem / nc, col = rem % nc;
    const int off = row * nc + tc_pos(row, col / 4, P) * 4 + col % 4;
    const double2 v = Dc[e];
    out[blk * 2 * n2 + off] = __double2float_rn(v.x);
    out[blk * 2 * n2 + n2 + off] = __double2float_rn(v.y);
  }
}

// FP32 coarse vector (optionally times xscale[r]; the scaled vector also to vout) -> FP32 rows of
// tf32_xpitch(NRHS) floats.
template <int NRHS>
__global__ void xc_to_f32rows_kernel(const float2* __restrict__ x, float* __restrict__ X, long long rows,
                                     const double* __restrict__ xscale, float2* __restrict__ vout,
                                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int XP = 2 * NRHS + (NRHS % 8 == 0 ? 8 : 0);
  const long long total = rows * NRHS;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % NRHS);
    float2 v = x[e];
    if (xscale) {
      const float f = (float)xscale[r];
      v.x *= f;
      v.y *= f;
    }
    if (vout) vout[e] = v;
    *reinterpret_cast<float2*>(X + (e / NRHS) * XP + 2 * r) = v;
  }
}

template <int NRHS>
__global__ void __launch_bounds__(160, 1) apply_tf32_kernel(const TfApplyArgs a, const int* skip, int ns) {
  if (skip && *skip) return;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  ring_init(pp, ns, (int)(blockDim.x >> 5) - 1);
  __syncthreads();
  const Ring rg{pp, sm + kPipeBytes, ns, tf32_apply_chunk(a.g.nc, NRHS)};
  RingPos rp;
  apply_tf32_items<NRHS>(a, rg, blockIdx.x, a.g.Vc, gridDim.x, rp);
  if (threadIdx.x == 0) drain(pp, rp.c, ns);
}

template <int NRHS>
amg_status launch_apply_tf32(amg_coarse* h, const void* x, void* y, cudaStream_t st, const int* skip,
                             const double* xscale, void* vout) {
  const int nc = h->g.nc;
  const size_t xsite = (size_t)nc * tf32_xpitch(NRHS) * 4;
  if ((size_t)h->g.Vc * xsite > h->tf_xbytes) return AMG_ERR_INVALID_ARG;  // nrhs > max_nrhs
  xc_to_f32rows_kernel<NRHS><<<4 * amg_sm_count(), 256, 0, st>>>((const float2*)x, (float*)h->tf_x, h->g.Vc * nc, xscale,
                                                      (float2*)vout, skip);
  AMG_LAUNCH_CHECK();
  h->launches++;
  const int threads = 32 + 32 * ((nc + 15) / 16);
  const size_t chunk = tf32_apply_chunk(nc, NRHS);
  int ns = (int)((56 * 1024) / chunk);
  ns = ns < 2 ? 2 : (ns > 4 ? 4 : ns);
  const size_t smem = kPipeBytes + ns * chunk;
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  AMG_CUDA_TRY(cudaFuncSetAttribute(apply_tf32_kernel<NRHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_tf32_kernel<NRHS>, threads, smem));
  if (per_sm < 1) return AMG_ERR_UNSUPPORTED;
  const long long gmax = (long long)per_sm * amg_sm_count();
  const int grid = capped_grid(h, h->g.Vc, gmax);
  TfApplyArgs a{(const float*)h->Dtf, (const float*)h->tf_x, h->nbr, (float2*)y, h->err, h->g};
  apply_tf32_kernel<NRHS><<<grid, threads, smem, st>>>(a, skip, ns);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

size_t tc_xbytes_per_site(const Geom& g, int nrhs) { return (size_t)g.nc * tc_xunits(nrhs) * 16; }

template <int NRHS>
amg_status launch_apply_tc(amg_coarse* h, const void* x, void* y, cudaStream_t st, const int* skip,
                           const double* xscale, void* vout) {
  const int nc = h->g.nc;
  const size_t xsite = tc_xbytes_per_site(h->g, NRHS);
  if ((size_t)h->g.Vc * xsite > h->tc_xbytes) return AMG_ERR_INVALID_ARG;  // nrhs > max_nrhs
  xc_to_bf16_kernel<NRHS><<<4 * amg_sm_count(), 256, 0, st>>>((const float2*)x, (__nv_bfloat162*)h->tc_x, h->g.Vc * nc, xscale,
                                                   (float2*)vout, skip);
  AMG_LAUNCH_CHECK();
  h->launches++;
  const int threads = 32 + 32 * ((nc + 15) / 16);
  const size_t chunk = tc_apply_chunk(nc, NRHS);
  // a short ring: more CTAs per SM (each works through its chunks in order) beat deeper prefetch
  int ns = (int)((32 * 1024) / chunk);
  ns = ns < 2 ? 2 : (ns > 6 ? 6 : ns);
  const size_t smem = kPipeBytes + ns * chunk;
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  AMG_CUDA_TRY(cudaFuncSetAttribute(apply_tc_kernel<NRHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_tc_kernel<NRHS>, threads, smem));
  if (per_sm < 1) return AMG_ERR_UNSUPPORTED;
  const long long gmax = (long long)per_sm * amg_sm_count();
  const int grid = capped_grid(h, h->g.Vc, gmax);
  TcApplyArgs a{(const bf16*)h->Dtc, (const bf16*)h->tc_x, h->nbr, (float2*)y, h->err, h->g};
  apply_tc_kernel<NRHS><<<grid, threads, smem, st>>>(a, skip, ns);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

}  // namespace

amg_status amg_internal_tc_prepare(amg_coarse* h, cudaStream_t st) {
  if (h->p.link_prec == AMG_BF16) {
    if (h->g.nc % 8 || h->g.nc > 64) return AMG_ERR_UNSUPPORTED;
    const size_t n = (size_t)h->g.Vc * 9 * 2 * h->g.nc * h->g.nc;
    AMG_CUDA_TRY(cudaMalloc(&h->Dtc, n * sizeof(bf16)));
    dc_to_bf16_kernel<<<4 * amg_sm_count(), 256, 0, st>>>(h->Dc64, (bf16*)h->Dtc, h->g.nc, h->g.Vc * 9);
    AMG_LAUNCH_CHECK();
    // BF16 planes of the apply's input, sized for the largest supported column count <= max_nrhs
    const int nmax = h->p.max_nrhs >= 16 ? 16 : (h->p.max_nrhs + 3) / 4 * 4;
    h->tc_xbytes = (size_t)h->g.Vc * tc_xbytes_per_site(h->g, nmax);
    AMG_CUDA_TRY(cudaMalloc(&h->tc_x, h->tc_xbytes));
  }
  if (h->p.link_prec == AMG_FP32 && h->p.vec_prec == AMG_FP32 && h->g.nc % 8 == 0 && h->g.nc <= 64 &&
      h->p.max_nrhs >= 4 && !amg_internal_tc5_supported(h)) {
    // FP32 D_c for the multi-RHS tensor-core apply (3 x TF32) where the tcgen05 form does not fit
    const size_t n = (size_t)h->g.Vc * 9 * 2 * h->g.nc * h->g.nc;
    AMG_CUDA_TRY(cudaMalloc(&h->Dtf, n * sizeof(float)));
    dc_to_tf32_kernel<<<4 * amg_sm_count(), 256, 0, st>>>(h->Dc64, (float*)h->Dtf, h->g.nc, h->g.Vc * 9);
    AMG_LAUNCH_CHECK();
    const int nmax = h->p.max_nrhs >= 16 ? 16 : h->p.max_nrhs / 4 * 4;
    h->tf_xbytes = (size_t)h->g.Vc * h->g.nc * tf32_xpitch(nmax) * 4;
    AMG_CUDA_TRY(cudaMalloc(&h->tf_x, h->tf_xbytes));
  }
  if (h->p.max_nrhs >= 4 && amg_internal_tc5_supported(h)) AMG_TRY_INTERNAL(amg_internal_tc5_prepare(h, st));
  if (h->p.r_prec == AMG_BF16) {
    const Geom& g = h->g;
    if (g.ntv % 4 || g.Vb % 8) return AMG_ERR_UNSUPPORTED;
    const size_t n = (size_t)g.Vc * 2 * 2 * g.ntv * g.nagg;
    AMG_CUDA_TRY(cudaMalloc(&h->Rtc, n * sizeof(bf16)));
    r_to_tc_kernel<<<4 * amg_sm_count(), 256, 0, st>>>(h->R64, (bf16*)h->Rtc, g);
    AMG_LAUNCH_CHECK();
  }
  return AMG_OK;
}

void amg_internal_free_tc(amg_coarse* h) {
  amg_internal_free_tc5(h);
  cudaFree(h->Dtc);
  cudaFree(h->Rtc);
  cudaFree(h->tc_x);
  cudaFree(h->Dtf);
  cudaFree(h->tf_x);
  h->Dtc = h->Rtc = h->tc_x = h->Dtf = h->tf_x = nullptr;
}

amg_status amg_internal_export_stored(amg_coarse* h, double2* out) {
  if (!h->Dtc) return AMG_ERR_UNSUPPORTED;
  const size_t n = (size_t)h->g.Vc * 9 * h->g.nc * h->g.nc;
  double2* tmp = nullptr;
  AMG_CUDA_TRY(cudaMalloc(&tmp, n * sizeof(double2)));
  bf16_to_dc_kernel<<<4 * amg_sm_count(), 256, 0, h->last_stream>>>((const bf16*)h->Dtc, tmp, h->g.nc, h->g.Vc * 9);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->last_stream);
  if (e == cudaSuccess) e = cudaMemcpy(out, tmp, n * sizeof(double2), cudaMemcpyDefault);
  cudaFree(tmp);
  if (e != cudaSuccess) {
    amg_note_cuda_error(__FILE__, __LINE__, e);
    return AMG_ERR_CUDA;
  }
  return AMG_OK;
}

amg_status amg_internal_apply_tc(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s,
                                 const int* skip, const double* xscale, void* vout) {
  if (!h->Dtc) return AMG_ERR_UNSUPPORTED;
  switch (nrhs) {
    case 4: return launch_apply_tc<4>(h, xc, yc, s, skip, xscale, vout);
    case 8: return launch_apply_tc<8>(h, xc, yc, s, skip, xscale, vout);
    case 12: return launch_apply_tc<12>(h, xc, yc, s, skip, xscale, vout);
    case 16: return launch_apply_tc<16>(h, xc, yc, s, skip, xscale, vout);
    default: return AMG_ERR_UNSUPPORTED;
  }
}

amg_status amg_internal_apply_tf32(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s,
                                   const int* skip, const double* xscale, void* vout) {
  if (!h->Dtf) return AMG_ERR_UNSUPPORTED;
  switch (nrhs) {
    case 4: return launch_apply_tf32<4>(h, xc, yc, s, skip, xscale, vout);
    case 8: return launch_apply_tf32<8>(h, xc, yc, s, skip, xscale, vout);
    case 12: return launch_apply_tf32<12>(h, xc, yc, s, skip, xscale, vout);
    case 16: return launch_apply_tf32<16>(h, xc, yc, s, skip, xscale, vout);
    default: return AMG_ERR_UNSUPPORTED;
  }
}

amg_status amg_internal_restrict_tc(amg_coarse* h, const void* y, void* yc, int nrhs, cudaStream_t s) {
  if (!h->Rtc) return AMG_ERR_UNSUPPORTED;
  switch (nrhs) {
    case 4: return launch_rp_tc<4, true>(h, y, yc, s);
    case 8: return launch_rp_tc<8, true>(h, y, yc, s);
    case 12: return launch_rp_tc<12, true>(h, y, yc, s);
    case 16: return launch_rp_tc<16, true>(h, y, yc, s);
    default: return AMG_ERR_UNSUPPORTED;
  }
}

amg_status amg_internal_prolong_tc(amg_coarse* h, const void* xc, void* x, int nrhs, cudaStream_t s) {
  if (!h->Rtc) return AMG_ERR_UNSUPPORTED;
  switch (nrhs) {
    case 4: return launch_rp_tc<4, false>(h, xc, x, s);
    case 8: return launch_rp_tc<8, false>(h, xc, x, s);
    case 12: return launch_rp_tc<12, false>(h, xc, x, s);
    case 16: return launch_rp_tc<16, false>(h, xc, x, s);
    default: return AMG_ERR_UNSUPPORTED;
  }
}
