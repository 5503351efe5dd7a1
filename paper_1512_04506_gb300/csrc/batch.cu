// One persistent launch for a batch of coarse-grid corrections x_k = P_k D_ck R_k y_k over several
// lattices of different size (Alg. 2 with a single coarse-operator application; the persistent
// threads with synchronisation points of Sec. 3 become persistent CTAs with per-lattice phase
// counters).
//
// The host lists every job in phase order: all restriction jobs, then all coarse-operator jobs,
// then all prolongation jobs; a job is a run of consecutive blocks or coarse sites of one lattice.
// CTAs take jobs from a global atomic counter.  A phase-2 job of lattice k first waits until all
// phase-1 jobs of lattice k have completed, a phase-3 job until all phase-2 jobs of k have; since
// every job waits only on jobs that were handed out earlier, and a job that has been handed out
// belongs to a running CTA that never waits on a later job, the schedule cannot deadlock whatever
// the number of resident CTAs.  Waits are bounded (about one second of clock cycles): a wait that
// runs out sets AMG_EBIT_TIMEOUT and an abort flag that makes every later wait return at once.
//
// Each lattice runs in its handle's precision.  FP32 lattices use the SIMT jobs below.  BF16
// lattices (R and D_c stored for the tensor cores, BF16 fine vectors, 4, 8, 12 or 16 right-hand
// sides) run the tensor-core bodies of tc_body.cuh through one bulk-copy ring per CTA that lives as
// long as the CTA; their restriction writes y_c directly as the BF16 rows the tensor-core apply
// reads, and the apply writes D_c y_c in FP32 for the prolongation.
//
// The launch issues only a memset and a kernel, so it can be captured in a CUDA graph once the
// work buffer exists (it is allocated by the first call).  amg_batch_autotune times candidate
// launch shapes (CTAs per SM x ring stages, or x threads per CTA when no lattice uses the tensor
// cores) on the caller's data and keeps the fastest.
#include "tc_body.cuh"

#include <vector>

namespace {
using namespace amgtc;

constexpr int kMaxLat = 8;
constexpr long long kBatchWaitCycles = 2000000000LL;
constexpr int kBatchThreads = 160;  // one producer warp + four consumer warps

struct LatDesc {
  Geom g;
  int tc;            // 1: BF16 tensor-core jobs, 0: FP32 SIMT jobs
  int nrhs;
  int ipj[3];        // blocks / sites per job of each phase
  const float2* R;   // FP32: [Vc][2][ntv][6Vb]
  const float2* D;   // FP32: apply layout [Vc][9][nc col][nc row]
  const int* nbr;    // [Vc][9]
  const float2* y;   // FP32 fine input  [V][12][nrhs]
  float2* x;         // FP32 fine output [V][12][nrhs]
  float2* yc;        // coarse scratch R y (FP32 lattices)
  float2* zc;        // coarse scratch D_c R y (FP32, both kinds)
  const bf16* Rtc;   // BF16: tensor-core R
  const bf16* Dtc;   // BF16: tensor-core D_c
  const void* ybf;   // BF16 fine input
  void* xbf;         // BF16 fine output
  __nv_bfloat162* rows;  // BF16: R y as the apply's BF16 rows
};

struct BatchArgs {
  LatDesc lat[kMaxLat];
  int nlat;
  const unsigned* jobs;  // (phase << 28) | (lattice << 24) | first item
  int njobs;
  unsigned* counters;    // [0] job counter, [1] abort, [2 + 3 k + p] completed jobs of phase p of k
  const int* need;       // [3 k + p] jobs of phase p of lattice k
  unsigned* err;
  int ns;                // ring stages
  unsigned stride;       // bytes per ring stage
};

__device__ inline unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

template <int NR>
__device__ void restrict_job(const LatDesc& L, long long blk, int r0, float2* sm) {
  const Geom& g = L.g;
  const int nagg = g.nagg, ntv = g.ntv, Vb = (int)g.Vb, ld = L.nrhs;
  float2* ys = sm;  // [2][nagg][NR]
  const long long origin = block_origin(g, blk);
  for (int e = threadIdx.x; e < Vb * 12 * NR; e += blockDim.x) {
    const int sl = e / (12 * NR), rem = e % (12 * NR), dof = rem / NR, r = rem % NR;
    const long long site = block_site_fast(g, origin, sl);
    ys[((size_t)(dof / 6) * nagg + sl * 6 + dof % 6) * NR + r] = L.y[(site * 12 + dof) * ld + r0 + r];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int row = warp; row < 2 * ntv; row += nw) {
    const float2* Rrow = L.R + (blk * 2 * ntv + row) * (long long)nagg;
    const float2* yh = ys + (size_t)(row / ntv) * nagg * NR;
    float2 acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int q = lane; q < nagg / 2; q += 32) {
      const float4 v = __ldcs(reinterpret_cast<const float4*>(Rrow) + q);
      const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
      // y of dofs 2q, 2q+1 for all NR right-hand sides: 2 NR consecutive values, 16-byte loads
      const float4* yp = reinterpret_cast<const float4*>(yh + (size_t)(2 * q) * NR);
#pragma unroll
      for (int u = 0; u < NR; ++u) {
        const float4 yy = yp[u];
        const int r = (2 * u) % NR;
        const bool second = 2 * u >= NR;  // entries 2u, 2u+1 of the run: dof 2q or 2q+1
        cfma(acc[r], second ? v1 : v0, make_float2(yy.x, yy.y));
        cfma(acc[r + 1 < NR ? r + 1 : 0], NR == 1 ? v1 : (second ? v1 : v0), make_float2(yy.z, yy.w));
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      float2 s = acc[r];
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) L.yc[(blk * 2 * ntv + row) * ld + r0 + r] = s;
    }
  }
  __syncthreads();
}

template <int NR>
__device__ void apply_job(const LatDesc& L, long long i, int r0, float2* sm) {
  const Geom& g = L.g;
  const int nc = g.nc, K = 9 * nc, Gc = nc / 2, ld = L.nrhs;
  const int G = (int)(blockDim.x / Gc) < nc ? (int)(blockDim.x / Gc) : nc;
  float2* xs = sm;              // [K][NR]
  float2* red = xs + K * NR;    // [G][nc][NR]
  for (int e = threadIdx.x; e < K * NR; e += blockDim.x) {
    const int k = e / NR, r = e % NR, d = k / nc, b = k % nc;
    xs[e] = L.yc[((long long)L.nbr[i * 9 + d] * nc + b) * ld + r0 + r];
  }
  __syncthreads();
  const int t = threadIdx.x, rc = t % Gc, grp = t / Gc;
  float2 acc[2][NR];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[q][r] = make_float2(0.f, 0.f);
  if (grp < G) {
    const float4* base = reinterpret_cast<const float4*>(L.D + i * (long long)K * nc) + rc;
#pragma unroll 4
    for (int k = grp; k < K; k += G) {
      const float4 v = __ldcs(base + (long long)k * Gc);
      const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        cfma(acc[0][r], v0, xs[k * NR + r]);
        cfma(acc[1][r], v1, xs[k * NR + r]);
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < NR; ++r) red[((size_t)grp * nc + 2 * rc + q) * NR + r] = acc[q][r];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nc * NR; e += blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int gg = 0; gg < G; ++gg) {
      const float2 v = red[(size_t)gg * nc * NR + e];
      s.x += v.x;
      s.y += v.y;
    }
    L.zc[(i * nc + e / NR) * ld + r0 + e % NR] = s;
  }
  __syncthreads();
}

template <int NR>
__device__ void prolong_job(const LatDesc& L, long long blk, int r0, float2* sm) {
  const Geom& g = L.g;
  const int nagg = g.nagg, ntv = g.ntv, tpa = nagg / 2, ld = L.nrhs;
  float2* xs = sm;  // [2 ntv][NR]
  const long long origin = block_origin(g, blk);
  for (int e = threadIdx.x; e < 2 * ntv * NR; e += blockDim.x)
    xs[e] = L.zc[(blk * 2 * ntv + e / NR) * ld + r0 + e % NR];
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * tpa; t += blockDim.x) {
    const int hh = t / tpa, n0 = (t % tpa) * 2;
    const float4* Rp = reinterpret_cast<const float4*>(L.R + (blk * 2 + hh) * (long long)ntv * nagg + n0);
    const float2* xh = xs + hh * ntv * NR;
    float2 acc[2][NR];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[q][r] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int j = 0; j < ntv; ++j) {
      const float4 v = __ldcs(Rp + (long long)j * (nagg / 2));
      const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        cfmac(acc[0][r], v0, xh[j * NR + r]);
        cfmac(acc[1][r], v1, xh[j * NR + r]);
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int n = n0 + q, sl = n / 6;
      const long long site = block_site_fast(g, origin, sl);
#pragma unroll
      for (int r = 0; r < NR; ++r) L.x[(site * 12 + hh * 6 + n % 6) * ld + r0 + r] = acc[q][r];
    }
  }
  __syncthreads();
}

template <int NR>
__device__ void run_job(const LatDesc& L, int phase, long long item, int r0, float2* sm) {
  if (phase == 0) restrict_job<NR>(L, item, r0, sm);
  else if (phase == 1) apply_job<NR>(L, item, r0, sm);
  else prolong_job<NR>(L, item, r0, sm);
}

// out of line in the tensor-core kernel, where inlining it would raise the register count of
// the whole kernel
template <int NR>
__device__ __noinline__ void run_job_outlined(const LatDesc& L, int phase, long long item, int r0, float2* sm) {
  run_job<NR>(L, phase, item, r0, sm);
}

// The ring position goes in and out by value so that it stays in registers inside the call.
template <int NRHS>
__device__ __noinline__ RingPos tc_job(const LatDesc& L, int phase, long long i0, long long i1, const Ring rg,
                                       RingPos rp, unsigned* err) {
  if (phase == 0) {
    const TcRPArgs a{L.Rtc, L.ybf, nullptr, L.rows, false, err, L.g};
    restrict_tc_items<NRHS>(a, rg, i0, i1, 1, rp);
  } else if (phase == 1) {
    const TcApplyArgs a{L.Dtc, reinterpret_cast<const bf16*>(L.rows), L.nbr, L.zc, err, L.g};
    apply_tc_items<NRHS>(a, rg, i0, i1, 1, rp);
  } else {
    const TcRPArgs a{L.Rtc, L.zc, L.xbf, nullptr, false, err, L.g};
    prolong_tc_items<NRHS>(a, rg, i0, i1, 1, rp);
  }
  return rp;
}

// TC: the batch holds tensor-core lattices (160 threads: one producer warp, four consumer warps);
// otherwise only SIMT jobs run and the thread count is free (autotuned).
template <bool TC>
__global__ void __launch_bounds__(TC ? kBatchThreads : 512, TC ? 4 : 1) batch_kernel(const BatchArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ unsigned job_s;
  __shared__ int ok_s;
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  if (TC) ring_init(pp, a.ns, (int)(blockDim.x >> 5) - 1);
  else if (threadIdx.x == 0) pp->abort = 0;
  __syncthreads();
  const Ring rg{pp, sm + kPipeBytes, a.ns, a.stride};
  float2* scratch = reinterpret_cast<float2*>(sm + kPipeBytes);  // SIMT jobs (the ring is idle then)
  volatile unsigned* abort_flag = a.counters + 1;
  RingPos rp;  // chunks through the ring (tensor-core jobs)
  for (;;) {
    if (threadIdx.x == 0) job_s = atomicAdd(a.counters, 1u);
    __syncthreads();
    const unsigned jid = job_s;
    if (jid >= (unsigned)a.njobs) break;
    const unsigned code = a.jobs[jid];
    const int phase = (int)(code >> 28), k = (int)((code >> 24) & 15);
    const long long first = code & 0xFFFFFF;
    const LatDesc& L = a.lat[k];
    const long long last = first + L.ipj[phase] < L.g.Vc ? first + L.ipj[phase] : L.g.Vc;
    if (threadIdx.x == 0) {
      int ok = !pp->abort;
      if (ok && phase > 0) {
        const unsigned* done = a.counters + 2 + 3 * k + (phase - 1);
        const unsigned need = (unsigned)a.need[3 * k + phase - 1];
        const long long t0 = clock64();
        while (ld_acquire(done) < need) {
          if (*abort_flag) {
            ok = 0;
            break;
          }
          if (clock64() - t0 > kBatchWaitCycles) {
            atomicOr(a.err, AMG_EBIT_TIMEOUT);
            *abort_flag = 1;
            ok = 0;
            break;
          }
        }
        // the earlier phase's results (written by other CTAs) are read next, partly by bulk copies
        __threadfence();
        if (TC) fence_proxy_async_global();
      }
      ok_s = ok;
    }
    __syncthreads();
    if (ok_s) {
      if (TC && L.tc) {
        switch (L.nrhs) {
          case 4: rp = tc_job<4>(L, phase, first, last, rg, rp, a.err); break;
          case 8: rp = tc_job<8>(L, phase, first, last, rg, rp, a.err); break;
          case 12: rp = tc_job<12>(L, phase, first, last, rg, rp, a.err); break;
          default: rp = tc_job<16>(L, phase, first, last, rg, rp, a.err); break;
        }
      } else {
        for (long long item = first; item < last; ++item) {
          int r0 = 0;
          while (r0 < L.nrhs) {
            const int nr = L.nrhs - r0 >= 4 ? 4 : 1;
            if (TC) {
              if (nr == 4) run_job_outlined<4>(L, phase, item, r0, scratch);
              else run_job_outlined<1>(L, phase, item, r0, scratch);
            } else {
              if (nr == 4) run_job<4>(L, phase, item, r0, scratch);
              else run_job<1>(L, phase, item, r0, scratch);
            }
            r0 += nr;
          }
        }
      }
    }
    if (TC) fence_proxy_async_global();  // this job's stores may be read by bulk copies of a later job
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.counters + 2 + 3 * k + phase, 1u);
      if (pp->abort) *abort_flag = 1;
    }
  }
  if (TC && threadIdx.x == 0) drain(pp, rp.c, a.ns);
}

size_t simt_smem(const Geom& g, int nrhs, int threads) {
  const int NR = nrhs >= 4 ? 4 : 1;
  const size_t r = (size_t)2 * g.nagg * NR * sizeof(float2);
  const int G = threads / (g.nc / 2) < g.nc ? threads / (g.nc / 2) : g.nc;
  const size_t ap = ((size_t)9 * g.nc * NR + (size_t)G * g.nc * NR) * sizeof(float2);
  const size_t p = (size_t)2 * g.ntv * NR * sizeof(float2);
  size_t m = r > ap ? r : ap;
  return m > p ? m : p;
}

// A lattice runs on the tensor cores when its R, D_c and vectors are all BF16 (prepare checks the
// column count).
bool tc_lattice(const amg_coarse* h) {
  return h->p.r_prec == AMG_BF16 && h->p.link_prec == AMG_BF16 && h->p.vec_prec == AMG_BF16;
}

struct Prepared {
  BatchArgs a;
  size_t smem;
  bool tc;  // some lattice runs on the tensor cores
};

amg_status prepare(amg_coarse* const* hs, int n, const void* const* y, void* const* x, const int* nrhs,
                   cudaStream_t st, int ns, int threads, Prepared* out) {
  if (n > kMaxLat) return AMG_ERR_UNSUPPORTED;
  BatchWork& bw = hs[0]->bw;
  // items per job: tensor-core restriction / prolongation 2 blocks, apply 8 sites; SIMT 1
  auto ipj = [&](int k, int p) { return tc_lattice(hs[k]) ? (p == 1 ? 8 : 2) : 1; };
  // layout of the work buffer: counters | need | jobs | per lattice coarse scratch
  size_t njobs = 0, coarse_bytes = 0;
  for (int k = 0; k < n; ++k) {
    const amg_coarse* h = hs[k];
    const bool tc = tc_lattice(h);
    if (tc) {
      if (!h->Rtc || !h->Dtc) return AMG_ERR_UNSUPPORTED;
      if (nrhs[k] != 4 && nrhs[k] != 8 && nrhs[k] != 12 && nrhs[k] != 16) return AMG_ERR_UNSUPPORTED;
    } else if (h->p.r_prec != AMG_FP32 || h->p.link_prec != AMG_FP32 || h->p.vec_prec != AMG_FP32) {
      return AMG_ERR_UNSUPPORTED;
    }
    if (h->g.Vc >= (1 << 24) || h->g.nc % 2) return AMG_ERR_UNSUPPORTED;
    for (int p = 0; p < 3; ++p) njobs += (size_t)((h->g.Vc + ipj(k, p) - 1) / ipj(k, p));
    const size_t vc = ((size_t)h->g.Vc * h->g.nc * nrhs[k] * sizeof(float2) + 255) / 256 * 256;
    const size_t rows = ((size_t)h->g.Vc * h->g.nc * tc_xunits(nrhs[k]) * 16 + 255) / 256 * 256;
    coarse_bytes += tc ? vc + rows : 2 * vc;
  }
  const size_t head = 256 + 256 + (njobs * sizeof(unsigned) + 255) / 256 * 256;
  const size_t need_bytes = head + coarse_bytes;
  if (need_bytes > bw.bytes) {
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(bw.buf);
    bw.buf = nullptr;
    bw.bytes = 0;
    AMG_CUDA_TRY(cudaMalloc(&bw.buf, need_bytes));
    bw.bytes = need_bytes;
    bw.sig = 0;
  }
  unsigned char* base = (unsigned char*)bw.buf;
  BatchArgs a{};
  a.nlat = n;
  a.counters = (unsigned*)base;
  a.need = (const int*)(base + 256);
  a.jobs = (const unsigned*)(base + 512);
  a.njobs = (int)njobs;
  a.err = hs[0]->err;
  a.ns = ns;
  size_t off = head;
  std::vector<int> need(3 * kMaxLat, 0);
  std::vector<unsigned> jobs;
  jobs.reserve(njobs);
  for (int phase = 0; phase < 3; ++phase)
    for (int k = 0; k < n; ++k)
      for (long long it = 0; it < hs[k]->g.Vc; it += ipj(k, phase)) {
        jobs.push_back(((unsigned)phase << 28) | ((unsigned)k << 24) | (unsigned)it);
        need[3 * k + phase]++;
      }
  size_t simt = 0;
  unsigned stride = 0;
  unsigned long long sig = 1469598103934665603ull;  // FNV-1a over the batch description
  for (int k = 0; k < n; ++k) {
    const amg_coarse* h = hs[k];
    LatDesc& L = a.lat[k];
    L.g = h->g;
    L.tc = tc_lattice(h) ? 1 : 0;
    L.nrhs = nrhs[k];
    for (int p = 0; p < 3; ++p) L.ipj[p] = ipj(k, p);
    L.nbr = h->nbr;
    const size_t vc = ((size_t)h->g.Vc * h->g.nc * nrhs[k] * sizeof(float2) + 255) / 256 * 256;
    if (L.tc) {
      L.Rtc = (const bf16*)h->Rtc;
      L.Dtc = (const bf16*)h->Dtc;
      L.ybf = y[k];
      L.xbf = x[k];
      L.zc = (float2*)(base + off);
      L.rows = (__nv_bfloat162*)(base + off + vc);
      off += vc + ((size_t)h->g.Vc * h->g.nc * tc_xunits(nrhs[k]) * 16 + 255) / 256 * 256;
      const unsigned ch[3] = {tc_restrict_chunk(h->g.ntv, nrhs[k]), tc_apply_chunk(h->g.nc, nrhs[k]),
                              tc_prolong_chunk(h->g.ntv)};
      for (int p = 0; p < 3; ++p) stride = ch[p] > stride ? ch[p] : stride;
    } else {
      L.R = (const float2*)h->Rq;
      L.D = (const float2*)h->Dq;
      L.y = (const float2*)y[k];
      L.x = (float2*)x[k];
      L.yc = (float2*)(base + off);
      L.zc = (float2*)(base + off + vc);
      off += 2 * vc;
      const size_t sm = simt_smem(h->g, nrhs[k], threads);
      simt = sm > simt ? sm : simt;
    }
    if (k == 0) need[0] += bw.test_extra_need;
    sig = (sig ^ (unsigned long long)(uintptr_t)h) * 1099511628211ull;
    sig = (sig ^ (unsigned long long)nrhs[k]) * 1099511628211ull;
  }
  a.stride = stride;
  sig = (sig ^ (unsigned long long)bw.test_extra_need) * 1099511628211ull;
  if (bw.sig != sig) {  // job list and phase counts only change with the batch description
    AMG_CUDA_TRY(cudaMemcpyAsync((void*)a.need, need.data(), need.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    AMG_CUDA_TRY(cudaMemcpyAsync((void*)a.jobs, jobs.data(), jobs.size() * sizeof(unsigned), cudaMemcpyHostToDevice, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    bw.sig = sig;
  }
  const size_t ring = (size_t)ns * stride;
  const size_t smem = kPipeBytes + (ring > simt ? ring : simt);
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  out->a = a;
  out->smem = smem;
  out->tc = stride > 0;
  return AMG_OK;
}

bool batch_has_tc(amg_coarse* const* hs, int n) {
  for (int k = 0; k < n; ++k)
    if (tc_lattice(hs[k])) return true;
  return false;
}

amg_status launch(const Prepared& pr, int threads, int per_sm, cudaStream_t st, amg_coarse* h0) {
  auto kern = pr.tc ? batch_kernel<true> : batch_kernel<false>;
  if (pr.tc) threads = kBatchThreads;
  AMG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pr.smem));
  int occ = 0;
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, pr.smem));
  if (occ < 1) return AMG_ERR_UNSUPPORTED;
  if (per_sm > occ) per_sm = occ;
  const long long resident = (long long)per_sm * amg_sm_count();
  AMG_CUDA_TRY(cudaMemsetAsync(pr.a.counters, 0, 256, st));
  kern<<<capped_grid(h0, resident, resident), threads, pr.smem, st>>>(pr.a);
  AMG_LAUNCH_CHECK();
  h0->launches++;
  return AMG_OK;
}

}  // namespace

amg_status amg_internal_batch(amg_coarse* const* hs, int n, const void* const* y, void* const* x, const int* nrhs,
                              cudaStream_t s) {
  BatchWork& bw = hs[0]->bw;
  const bool tc = batch_has_tc(hs, n);
  const int threads = tc ? kBatchThreads : (bw.threads ? bw.threads : 256);
  const int ns = bw.ns ? bw.ns : 3;
  const int per_sm = bw.per_sm ? bw.per_sm : (tc ? 4 : 2);
  Prepared pr;
  amg_status st = prepare(hs, n, y, x, nrhs, s, tc ? ns : 0, threads, &pr);
  if (st != AMG_OK) return st;
  return launch(pr, threads, per_sm, s, hs[0]);
}

extern "C" amg_status amg_batch_autotune(const amg_handle* hs, int n, const void* const* d_y, void* const* d_x,
                                         const int* nrhs, void* stream, double* best_ms) {
  if (!hs || n < 1 || !d_y || !d_x || !nrhs) return AMG_ERR_INVALID_ARG;
  for (int k = 0; k < n; ++k)
    if (!hs[k] || !d_y[k] || !d_x[k] || nrhs[k] < 1 || nrhs[k] > hs[k]->p.max_nrhs) return AMG_ERR_INVALID_ARG;
  for (int k = 0; k < n; ++k)
    if (hs[k]->level != 1) return AMG_ERR_UNSUPPORTED;  // a level-2 handle has no fine lattice
  cudaStream_t st = (cudaStream_t)stream;
  amg_coarse* const* H = const_cast<amg_coarse* const*>(hs);
  // tensor-core batches: ring stages x CTAs per SM; SIMT-only batches: threads per CTA x CTAs per SM
  const bool tc = batch_has_tc(H, n);
  const int cand_a[3] = {2, 3, 4}, cand_threads[3] = {128, 256, 512};
  const int cand_per_sm[4] = {1, 2, 3, 4};
  float best = 1e30f;
  int ba = tc ? 3 : 256, bp = tc ? 3 : 2;
  cudaEvent_t e0, e1;
  AMG_CUDA_TRY(cudaEventCreate(&e0));
  AMG_CUDA_TRY(cudaEventCreate(&e1));
  for (int ai = 0; ai < 3; ++ai)
    for (int pi = 0; pi < 4; ++pi) {
      const int ns = tc ? cand_a[ai] : 0, threads = tc ? kBatchThreads : cand_threads[ai];
      Prepared pr;
      if (prepare(H, n, d_y, d_x, nrhs, st, ns, threads, &pr) != AMG_OK) continue;
      if (launch(pr, threads, cand_per_sm[pi], st, H[0]) != AMG_OK) continue;  // warm-up
      float ms = 0, tot = 0;
      bool good = true;
      for (int rep = 0; rep < 3 && good; ++rep) {
        cudaEventRecord(e0, st);
        good = launch(pr, threads, cand_per_sm[pi], st, H[0]) == AMG_OK;
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        tot += ms;
      }
      if (good && tot / 3 < best) {
        best = tot / 3;
        ba = tc ? cand_a[ai] : cand_threads[ai];
        bp = cand_per_sm[pi];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (tc) H[0]->bw.ns = ba;
  else H[0]->bw.threads = ba;
  H[0]->bw.per_sm = bp;
  if (best_ms) *best_ms = best;
  for (int k = 0; k < n; ++k) H[k]->last_stream = st;
  return best < 1e30f ? AMG_OK : AMG_ERR_UNSUPPORTED;
}

extern "C" amg_status amg_batch_test_hook(amg_handle h0, int extra_need) {
  if (!h0 || extra_need < 0) return AMG_ERR_INVALID_ARG;
  h0->bw.test_extra_need = extra_need;
  h0->bw.sig = 0;
  return AMG_OK;
}
