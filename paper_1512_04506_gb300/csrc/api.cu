// The C ABI of libamg: argument validation, handle life cycle, exports.
#include "amg_internal.cuh"

#include <new>
#include <stdarg.h>
#include <stdio.h>
#include <vector>

static thread_local char g_last_error[256] = "";

void amg_note_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

void amg_note_cuda_error(const char* file, int line, cudaError_t e) {
  const char* base = strrchr(file, '/');
  snprintf(g_last_error, sizeof(g_last_error), "%s:%d: %s (%s)", base ? base + 1 : file, line,
           cudaGetErrorString(e), cudaGetErrorName(e));
}

int amg_sm_count() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  if (dev >= 64) dev = 63;
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev] = n;
  }
  return cache[dev];
}

namespace {

bool valid_prec(amg_prec p) { return p >= AMG_FP64 && p <= AMG_BF16; }

amg_status validate_params(const amg_params* p) {
  if (!p) return AMG_ERR_INVALID_ARG;
  long long Vb = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (p->L[mu] < 2 || p->B[mu] < 1 || p->L[mu] % p->B[mu]) return AMG_ERR_INVALID_ARG;
    if (p->L[mu] / p->B[mu] < 2) return AMG_ERR_INVALID_ARG;
    Vb *= p->B[mu];
  }
  if (p->ntv < 1 || p->ntv > AMG_MAX_NTV || p->ntv > 6 * Vb) return AMG_ERR_INVALID_ARG;
  if (p->max_nrhs < 1 || p->max_nrhs > 64) return AMG_ERR_INVALID_ARG;
  if (!valid_prec(p->link_prec) || !valid_prec(p->r_prec) || !valid_prec(p->vec_prec)) return AMG_ERR_INVALID_ARG;
  if (p->r_prec == AMG_FP16_SCALED || p->vec_prec == AMG_FP16_SCALED) return AMG_ERR_INVALID_ARG;
  if (p->setup_arith != AMG_SETUP_FP64 && p->setup_arith != AMG_SETUP_F32PAIR) return AMG_ERR_INVALID_ARG;
  // supported storage / vector combinations
  if (p->vec_prec == AMG_FP64) {
    if (p->link_prec != AMG_FP64 || p->r_prec != AMG_FP64) return AMG_ERR_UNSUPPORTED;
  } else if (p->vec_prec == AMG_FP32) {
    if (p->link_prec == AMG_FP64 || p->r_prec != AMG_FP32) return AMG_ERR_UNSUPPORTED;
  } else {  // BF16 fine vectors: tensor-core path
    if (p->r_prec != AMG_BF16 || p->link_prec != AMG_BF16) return AMG_ERR_UNSUPPORTED;
  }
  if (p->link_prec == AMG_FP16_SCALED && (p->ntv % 2)) return AMG_ERR_UNSUPPORTED;
  if (p->ntv > 32) return AMG_ERR_UNSUPPORTED;  // register tiles of the D_c assembly
  return AMG_OK;
}

Geom make_geom(const amg_params* p) {
  Geom g;
  g.V = g.Vb = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.L[mu] = p->L[mu];
    g.B[mu] = p->B[mu];
    g.Lc[mu] = p->L[mu] / p->B[mu];
    g.V *= p->L[mu];
    g.Vb *= p->B[mu];
  }
  g.Vc = g.V / g.Vb;
  g.ntv = p->ntv;
  g.nc = 2 * p->ntv;
  g.nagg = (int)(6 * g.Vb);
  return g;
}

void free_handle(amg_coarse* h) {
  if (!h) return;
  if (h->next) h->next->prev = nullptr;  // an attached level 2 / level 1 forgets this handle
  if (h->prev) h->prev->next = nullptr;
  cudaFree(h->l2work);
  cudaFree(h->clover);
  if (h->Rq != (void*)h->R64) cudaFree(h->Rq);
  cudaFree(h->R64);
  cudaFree(h->Dc64);
  cudaFree(h->Dq);
  cudaFree(h->Dscale);
  cudaFree(h->nbr);
  cudaFree(h->soff);
  cudaFree(h->Dinv64);
  cudaFree(h->Dinvq);
  cudaFree(h->eo_site);
  cudaFree(h->eo_tmp);
  cudaFree(h->err);
  cudaFree(h->sw.buf);
  if (h->sw.hflag) {
    cudaFreeHost(h->sw.hflag);
    for (int k = 0; k < SolveWork::kRing; ++k) cudaEventDestroy(h->sw.ev[k]);
  }
  cudaFree(h->bw.buf);
  cudaFree(h->xc_tmp);
  cudaFree(h->yc_tmp);
  amg_internal_free_tc(h);
  amg_internal_free_fine(h);
  delete h;
}

template <typename T>
amg_status dmalloc(T** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA;
  }
  return AMG_OK;
}

#define AMG_TRY(x)                  \
  do {                              \
    amg_status s_ = (x);            \
    if (s_ != AMG_OK) return s_;    \
  } while (0)

amg_status check_apply_args(amg_handle h, const void* a, const void* b, int nrhs) {
  if (!h || !a || !b) return AMG_ERR_INVALID_ARG;
  if (!aligned16(a) || !aligned16(b)) return AMG_ERR_INVALID_ARG;
  if (nrhs < 1 || nrhs > h->p.max_nrhs) return AMG_ERR_INVALID_ARG;
  return AMG_OK;
}

__global__ void dequantize_kernel(const void* Dq, const float* scale, int mode, double2* out, int nc,
                                  long long nblocks) {
  const long long n2 = (long long)nc * nc;
  const long long total = nblocks * n2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / n2;
    const int rem = (int)(e % n2), a = rem / nc, c = rem % nc;  // out[blk][a][c]
    const long long src = blk * n2 + (long long)c * nc + a;      // stored column-major
    double2 v;
    if (mode == 0) {
      v = ((const double2*)Dq)[src];
    } else if (mode == 1) {
      const float2 f = ((const float2*)Dq)[src];
      v = make_double2(f.x, f.y);
    } else {
      const __half2 hv = ((const __half2*)Dq)[src];
      const double s = scale[blk];
      v = make_double2((double)__half2float(hv.x) * s, (double)__half2float(hv.y) * s);
    }
    out[e] = v;
  }
}

}  // namespace

extern "C" {

amg_status amg_setup_coarse(const amg_params* p, const void* d_U, const void* d_tv, void* stream,
                            amg_handle* out) {
  if (!out) return AMG_ERR_INVALID_ARG;
  *out = nullptr;
  AMG_TRY(validate_params(p));
  if (!d_U || !d_tv || !aligned16(d_U) || !aligned16(d_tv)) return AMG_ERR_INVALID_ARG;
  amg_coarse* h = new (std::nothrow) amg_coarse();
  if (!h) return AMG_ERR_OOM;
  h->p = *p;
  h->g = make_geom(p);
  const Geom& g = h->g;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  amg_status s = AMG_OK;
  const size_t nR = (size_t)g.Vc * 2 * g.ntv * g.nagg;
  const size_t nD = (size_t)g.Vc * 9 * g.nc * g.nc;
#define AMG_TRY_H(x)      \
  do {                    \
    s = (x);              \
    if (s != AMG_OK) {    \
      free_handle(h);     \
      return s;           \
    }                     \
  } while (0)
  AMG_TRY_H(dmalloc(&h->clover, (size_t)g.V * 72 * sizeof(double2)));
  AMG_TRY_H(dmalloc(&h->R64, nR * sizeof(double2)));
  if (p->r_prec == AMG_FP64) h->Rq = h->R64;
  else if (p->r_prec == AMG_FP32) AMG_TRY_H(dmalloc(&h->Rq, nR * sizeof(float2)));
  AMG_TRY_H(dmalloc(&h->Dc64, nD * sizeof(double2)));
  if (p->link_prec == AMG_FP64) AMG_TRY_H(dmalloc(&h->Dq, nD * sizeof(double2)));
  else if (p->link_prec == AMG_FP32) AMG_TRY_H(dmalloc(&h->Dq, nD * sizeof(float2)));
  else if (p->link_prec == AMG_FP16_SCALED) {
    AMG_TRY_H(dmalloc(&h->Dq, nD * sizeof(__half2)));
    AMG_TRY_H(dmalloc(&h->Dscale, (size_t)g.Vc * 9 * sizeof(float)));
  }
  AMG_TRY_H(dmalloc(&h->nbr, (size_t)g.Vc * 9 * sizeof(int)));
  AMG_TRY_H(dmalloc(&h->soff, (size_t)g.Vb * sizeof(int)));
  {
    std::vector<int> so((size_t)g.Vb);
    for (int s = 0; s < (int)g.Vb; ++s) {
      const int bx = s % g.B[0], by = (s / g.B[0]) % g.B[1], bz = (s / (g.B[0] * g.B[1])) % g.B[2];
      const int bt = s / (g.B[0] * g.B[1] * g.B[2]);
      so[s] = (int)site_index(g.L, bx, by, bz, bt);
    }
    if (cudaMemcpy(h->soff, so.data(), so.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
      free_handle(h);
      return AMG_ERR_CUDA;
    }
    h->g.soff = h->soff;
  }
  AMG_TRY_H(dmalloc(&h->err, sizeof(unsigned)));
  {
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
    if (cudaMemcpy(h->nbr, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
      free_handle(h);
      return AMG_ERR_CUDA;
    }
  }
  if (cudaMemsetAsync(h->err, 0, sizeof(unsigned), st) != cudaSuccess) {
    free_handle(h);
    return AMG_ERR_CUDA;
  }
  s = amg_internal_setup(h, (const double2*)d_U, (const double2*)d_tv, st);
  if (s == AMG_OK || s == AMG_ERR_RANK_DEFICIENT) {
    *out = h;
    return s;
  }
  cudaStreamSynchronize(st);
  free_handle(h);
  return s;
#undef AMG_TRY_H
}

}  // extern "C"

amg_status amg_internal_rebuild(amg_coarse* h, const double2* U, const double2* tv, cudaStream_t st) {
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  amg_internal_free_tc(h);
  cudaFree(h->eo_site);
  cudaFree(h->Dinv64);
  cudaFree(h->Dinvq);
  cudaFree(h->eo_tmp);
  h->eo_site = nullptr;
  h->Dinv64 = nullptr;
  h->Dinvq = nullptr;
  h->eo_tmp = nullptr;
  h->eo_tmp_bytes = 0;
  h->bw.sig = 0;  // a cached batch job list may hold the old tensor-core copies
  AMG_CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(unsigned), st));
  return amg_internal_setup(h, U, tv, st);
}

extern "C" {

amg_status amg_restrict(amg_handle h, const void* d_y, void* d_yc, int nrhs, void* stream) {
  AMG_TRY(check_apply_args(h, d_y, d_yc, nrhs));
  if (h->level != 1) return AMG_ERR_UNSUPPORTED;  // a level-2 handle has no fine lattice
  h->last_stream = (cudaStream_t)stream;
  return amg_internal_restrict(h, d_y, d_yc, nrhs, (cudaStream_t)stream);
}

amg_status amg_coarse_apply(amg_handle h, const void* d_xc, void* d_yc, int nrhs, void* stream) {
  AMG_TRY(check_apply_args(h, d_xc, d_yc, nrhs));
  if (d_xc == d_yc) return AMG_ERR_INVALID_ARG;
  h->last_stream = (cudaStream_t)stream;
  return amg_internal_apply(h, d_xc, d_yc, nrhs, (cudaStream_t)stream);
}

amg_status amg_prolong(amg_handle h, const void* d_xc, void* d_x, int nrhs, void* stream) {
  AMG_TRY(check_apply_args(h, d_xc, d_x, nrhs));
  if (h->level != 1) return AMG_ERR_UNSUPPORTED;
  h->last_stream = (cudaStream_t)stream;
  return amg_internal_prolong(h, d_xc, d_x, nrhs, (cudaStream_t)stream);
}

amg_status amg_coarse_solve(amg_handle h, const void* d_b, void* d_x, int nrhs, double tol, int restart,
                            int max_applies, void* stream, double* info) {
  AMG_TRY(check_apply_args(h, d_b, d_x, nrhs));
  if (d_b == d_x || !(tol >= 0)) return AMG_ERR_INVALID_ARG;
  h->last_stream = (cudaStream_t)stream;
  return amg_internal_solve(h, d_b, d_x, nrhs, tol, restart, max_applies, (cudaStream_t)stream, info);
}

amg_status amg_cgc(amg_handle h, const void* d_y, void* d_x, int nrhs, double tol, int restart,
                   int max_applies, void* stream, double* info) {
  AMG_TRY(check_apply_args(h, d_y, d_x, nrhs));
  if (h->level != 1) return AMG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  const size_t bytes = (size_t)h->g.Vc * h->g.nc * nrhs * coarse_elem_bytes(h);
  if (bytes > h->tmp_bytes) {
    cudaStreamSynchronize(st);
    cudaFree(h->xc_tmp);
    cudaFree(h->yc_tmp);
    h->xc_tmp = h->yc_tmp = nullptr;
    h->tmp_bytes = 0;
    AMG_TRY(dmalloc(&h->xc_tmp, bytes));
    AMG_TRY(dmalloc(&h->yc_tmp, bytes));
    h->tmp_bytes = bytes;
  }
  AMG_TRY(amg_internal_restrict(h, d_y, h->yc_tmp, nrhs, st));
  AMG_TRY(amg_internal_solve(h, h->yc_tmp, h->xc_tmp, nrhs, tol, restart, max_applies, st, info));
  return amg_internal_prolong(h, h->xc_tmp, d_x, nrhs, st);
}

amg_status amg_batch_cgc(const amg_handle* hs, int n, const void* const* d_y, void* const* d_x, const int* nrhs,
                         void* stream) {
  if (!hs || n < 1 || !d_y || !d_x || !nrhs) return AMG_ERR_INVALID_ARG;
  for (int k = 0; k < n; ++k) {
    AMG_TRY(check_apply_args(hs[k], d_y[k], d_x[k], nrhs[k]));
    if (hs[k]->level != 1) return AMG_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < n; ++k) hs[k]->last_stream = (cudaStream_t)stream;
  return amg_internal_batch(const_cast<amg_coarse* const*>(hs), n, d_y, d_x, nrhs, (cudaStream_t)stream);
}

static amg_status copy_out(amg_handle h, void* out, const void* src, size_t bytes) {
  if (!h || !out) return AMG_ERR_INVALID_ARG;
  AMG_CUDA_TRY(cudaStreamSynchronize(h->last_stream));
  AMG_CUDA_TRY(cudaMemcpy(out, src, bytes, cudaMemcpyDefault));
  return AMG_OK;
}

amg_status amg_export_R(amg_handle h, void* out) {
  if (!h) return AMG_ERR_INVALID_ARG;
  return copy_out(h, out, h->R64, (size_t)h->g.Vc * 2 * h->g.ntv * h->g.nagg * sizeof(double2));
}

amg_status amg_export_Dc(amg_handle h, void* out) {
  if (!h) return AMG_ERR_INVALID_ARG;
  return copy_out(h, out, h->Dc64, (size_t)h->g.Vc * 9 * h->g.nc * h->g.nc * sizeof(double2));
}

amg_status amg_export_clover(amg_handle h, void* out) {
  if (!h) return AMG_ERR_INVALID_ARG;
  if (h->level != 1) return AMG_ERR_UNSUPPORTED;
  return copy_out(h, out, h->clover, (size_t)h->g.V * 72 * sizeof(double2));
}

amg_status amg_export_Dc_stored(amg_handle h, void* out) {
  if (!h || !out) return AMG_ERR_INVALID_ARG;
  const size_t n = (size_t)h->g.Vc * 9 * h->g.nc * h->g.nc;
  if (h->p.link_prec == AMG_BF16) return amg_internal_export_stored(h, (double2*)out);
  double2* tmp = nullptr;
  AMG_TRY(dmalloc(&tmp, n * sizeof(double2)));
  const int mode = h->p.link_prec == AMG_FP64 ? 0 : (h->p.link_prec == AMG_FP32 ? 1 : 2);
  dequantize_kernel<<<1024, 256, 0, h->last_stream>>>(h->Dq, h->Dscale, mode, tmp, h->g.nc, h->g.Vc * 9);
  amg_status s = copy_out(h, out, tmp, n * sizeof(double2));
  cudaFree(tmp);
  return s;
}

amg_status amg_setup_timings(amg_handle h, double out_ms[4]) {
  if (!h || !out_ms) return AMG_ERR_INVALID_ARG;
  for (int k = 0; k < 4; ++k) out_ms[k] = h->setup_ms[k];
  return AMG_OK;
}

amg_status amg_kernel_launches(amg_handle h, unsigned long long* out) {
  if (!h || !out) return AMG_ERR_INVALID_ARG;
  *out = h->launches;
  return AMG_OK;
}

amg_status amg_sync_status(amg_handle h) {
  if (!h) return AMG_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return AMG_ERR_CUDA;
  unsigned e = 0;
  if (cudaMemcpy(&e, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return AMG_ERR_CUDA;
  if (e && cudaMemset(h->err, 0, sizeof(unsigned)) != cudaSuccess) return AMG_ERR_CUDA;  // reported once
  if (e & AMG_EBIT_TIMEOUT) return AMG_ERR_TIMEOUT;
  if (e & AMG_EBIT_RANK) return AMG_ERR_RANK_DEFICIENT;
  if (e & AMG_EBIT_NONFINITE) return AMG_ERR_NONFINITE;
  if (e) return AMG_ERR_CUDA;
  return AMG_OK;
}

amg_status amg_destroy(amg_handle h) {
  if (!h) return AMG_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->last_stream);
  free_handle(h);
  return AMG_OK;
}

const char* amg_last_error(void) { return g_last_error; }

const char* amg_status_string(amg_status s) {
  switch (s) {
    case AMG_OK: return "ok";
    case AMG_ERR_INVALID_ARG: return "invalid argument";
    case AMG_ERR_UNSUPPORTED: return "unsupported configuration";
    case AMG_ERR_OOM: return "out of device memory";
    case AMG_ERR_CUDA: return "CUDA error";
    case AMG_ERR_TIMEOUT: return "device wait timed out";
    case AMG_ERR_RANK_DEFICIENT: return "test vectors are rank deficient on an aggregate";
    case AMG_ERR_NONFINITE: return "non-finite value";
  }
  return "unknown status";
}

}  // extern "C"
