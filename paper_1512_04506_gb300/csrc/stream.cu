// Streaming kernels for the three HBM-bound steps of the coarse-grid correction (Alg. 2):
// restriction y_c = R y (Eq. R, Alg. 6), coarse operator y_c = D_c x_c and prolongation
// x = P x_c with P = R^dagger.
//
// The coarse operator (and the FP64 prolongation) is persistent and TMA-fed; the restriction and
// the FP32 prolongation are plain one-CTA-per-block kernels (measured faster for their access
// patterns, see restrict_kernel and prolong_pair_kernel).
// In the TMA-fed kernels each CTA is persistent over work items (blocks for P, coarse sites for
// D_c), taken in strided order so that the CTAs in flight read neighbouring items.  Warp 0 is
// the producer: one lane streams the item's matrix into a ring of shared-memory stages with
// cp.async.bulk, each stage guarded by a "full" mbarrier (transaction bytes) and an "empty"
// mbarrier (consumer release).  The other warps consume the stages from shared memory.  The
// producer runs ahead across item boundaries, so the stream never stops while the consumers
// stage the small vectors of the next item.  Every wait is bounded (about one second of clock
// cycles); a wait that runs out sets AMG_EBIT_TIMEOUT, makes the CTA skip the rest of its work,
// and the producer still waits (bounded) for the copies it has issued before the CTA exits.
#include "amg_internal.cuh"
#include "pipe.cuh"

#include <type_traits>

namespace {
using namespace amgpipe;

template <typename T> struct Acc;
template <> struct Acc<double2> { using type = double2; };
template <> struct Acc<float2> { using type = float2; };
template <> struct Acc<__half2> { using type = float2; };

// 16 bytes of shared memory as CPL complex values of the accumulation type.
template <typename T> struct Vec16;
template <> struct Vec16<double2> {
  static constexpr int CPL = 1;
  __device__ static void ld(const double2* p, double2 (&v)[1]) { v[0] = *p; }
};
template <> struct Vec16<float2> {
  static constexpr int CPL = 2;
  __device__ static void ld(const float2* p, float2 (&v)[2]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = make_float2(t.x, t.y);
    v[1] = make_float2(t.z, t.w);
  }
};
template <> struct Vec16<__half2> {
  static constexpr int CPL = 4;
  __device__ static void ld(const __half2* p, float2 (&v)[4]) {
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    const unsigned u[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __half2 hv;
      memcpy(&hv, &u[k], 4);
      v[k] = __half22float2(hv);
    }
  }
};

// n consecutive complex values from 16-byte aligned shared memory, with 16-byte loads.
template <typename AT, int n>
__device__ inline void load_run(const AT* p, AT (&v)[n]) {
  if constexpr (sizeof(AT) == 8 && n % 2 == 0) {
#pragma unroll
    for (int u = 0; u < n / 2; ++u) {
      const float4 t = reinterpret_cast<const float4*>(p)[u];
      v[2 * u] = AT{t.x, t.y};
      v[2 * u + 1] = AT{t.z, t.w};
    }
  } else {
#pragma unroll
    for (int u = 0; u < n; ++u) v[u] = p[u];
  }
}

// 16 bytes of global memory (read once, not kept in L1) as CPL complex values.
template <typename T> struct Ld16;
template <> struct Ld16<double2> {
  __device__ static void ld(const double2* p, double2 (&v)[1]) { v[0] = __ldcs(p); }
};
template <> struct Ld16<float2> {
  __device__ static void ld(const float2* p, float2 (&v)[2]) {
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = make_float2(t.x, t.y);
    v[1] = make_float2(t.z, t.w);
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

// One complex value global -> shared without a register round trip (cp.async, 8 or 16 bytes).
__device__ inline void cp_async_elem(float2* dst, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ inline void cp_async_elem(double2* dst, const double2* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename AT>
__device__ inline AT scaled(AT v, double f) {
  using RT = decltype(v.x);
  return AT{v.x * (RT)f, v.y * (RT)f};
}

// ------------------------------------------------------------------ coarse operator
// Item = coarse site i; chunk d (0..8) = stencil block D_c[i][d], column-major, nc*nc entries.
// Consumers stage X[d][b] = s_d * x(nbr(i, d))[b] (s_d the FP16 block scale; x optionally times
// xscale[r], in which case the consumers of direction 0 also store the scaled own vector to
// vout), then thread (rc, grp) accumulates rows rc*CPL.. over columns b = grp, grp + G, ...
template <typename LT, int NR>
struct ApplyArgs {
  using AT = typename Acc<LT>::type;
  const LT* D;
  const float* dscale;
  const int* nbr;
  const AT* x;
  AT* y;
  AT* vout;
  const double* xscale;
  const int* skip;
  unsigned* err;
  Geom g;
  int ld, r0, ns, G;
};

template <typename LT, int NR>
__global__ void __launch_bounds__(288) apply_tma_kernel(const ApplyArgs<LT, NR> a) {
  using AT = typename Acc<LT>::type;
  constexpr int CPL = Vec16<LT>::CPL;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int nc = a.g.nc, K = 9 * nc, ns = a.ns;
  const unsigned chunk = (unsigned)(nc * nc * sizeof(LT));
  unsigned char* stages = sm + kPipeBytes;
  AT* xs = reinterpret_cast<AT*>(stages + (size_t)ns * chunk);  // [2][K][NR]
  AT* red = xs + (size_t)2 * K * NR;
  const int ncw = (blockDim.x - 32) >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&pp->full[s], 1);
      mbar_init(&pp->empty[s], ncw);
    }
    pp->abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const long long Vc = a.g.Vc;
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      long long c = 0;
      for (long long i = blockIdx.x; i < Vc && !pp->abort; i += gridDim.x) {
        for (int d = 0; d < 9; ++d, ++c) {
          const int s = (int)(c % ns);
          const long long q = c / ns;
          if (c >= ns && !wait_phase(&pp->empty[s], (unsigned)((q - 1) & 1), pp)) {
            abort_cta(pp, a.err);
            break;
          }
          mbar_expect_tx(&pp->full[s], chunk);
          bulk_load_hint(stages + (size_t)s * chunk, a.D + (i * 9 + d) * (long long)nc * nc, chunk, &pp->full[s],
                         l2_evict_first_policy());
        }
      }
      drain(pp, c, ns);
    }
    return;
  }
  const int t = threadIdx.x - 32, nct = blockDim.x - 32;
  const int Gc = nc / CPL, rc = t % Gc, grp = t / Gc;
  // Neighbour vectors of site i, gathered asynchronously one site ahead into the other buffer;
  // each thread later scales exactly the elements it gathered (no barrier needed in between).
  auto gather = [&](long long i, AT* buf) {
    for (int e = t; e < K * NR; e += nct) {
      const int k = e / NR, r = e % NR, d = k / nc, b = k % nc;
      const long long j = a.nbr[i * 9 + d];
      cp_async_elem(buf + e, a.x + (j * nc + b) * a.ld + a.r0 + r);
    }
    cp_async_commit();
  };
  auto finish = [&](long long i, AT* buf) {
    cp_async_wait_all();
    if (!a.xscale && !a.dscale) return;
    for (int e = t; e < K * NR; e += nct) {
      const int k = e / NR, r = e % NR, d = k / nc, b = k % nc;
      AT v = buf[e];
      if (a.xscale) {
        v = scaled(v, a.xscale[a.r0 + r]);
        if (d == 0 && a.vout) a.vout[(i * nc + b) * a.ld + a.r0 + r] = v;
      }
      if (a.dscale) v = scaled(v, (double)a.dscale[i * 9 + d]);
      buf[e] = v;
    }
  };
  long long c = 0;
  int it = 0;
  if (blockIdx.x < Vc) {
    gather(blockIdx.x, xs);
    finish(blockIdx.x, xs);
  }
  consumer_sync(nct);
  for (long long i = blockIdx.x; i < Vc; i += gridDim.x, ++it) {
    AT* xcur = xs + (size_t)(it & 1) * K * NR;
    AT* xnext = xs + (size_t)((it + 1) & 1) * K * NR;
    const long long inext = i + gridDim.x;
    if (inext < Vc) gather(inext, xnext);
    AT acc[CPL][NR];
#pragma unroll
    for (int q = 0; q < CPL; ++q)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[q][r] = AT{0, 0};
    for (int d = 0; d < 9; ++d, ++c) {
      const int s = (int)(c % ns);
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], (unsigned)((c / ns) & 1), pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      if (ok && grp < a.G) {
        const LT* blk = reinterpret_cast<const LT*>(stages + (size_t)s * chunk) + rc * CPL;
        const AT* xd = xcur + (size_t)d * nc * NR;
#pragma unroll 4
        for (int b = grp; b < nc; b += a.G) {
          AT v[CPL];
          Vec16<LT>::ld(blk + (size_t)b * nc, v);
#pragma unroll
          for (int q = 0; q < CPL; ++q)
#pragma unroll
            for (int r = 0; r < NR; ++r) cfma(acc[q][r], v[q], xd[b * NR + r]);
        }
      }
      __syncwarp();
      if ((t & 31) == 0) mbar_arrive(&pp->empty[s]);
    }
    if (grp < a.G)
#pragma unroll
      for (int q = 0; q < CPL; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) red[((size_t)grp * nc + rc * CPL + q) * NR + r] = acc[q][r];
    consumer_sync(nct);
    for (int e = t; e < nc * NR; e += nct) {
      AT sum = AT{0, 0};
      for (int gg = 0; gg < a.G; ++gg) {
        const AT v = red[(size_t)gg * nc * NR + e];
        sum.x += v.x;
        sum.y += v.y;
      }
      a.y[(i * nc + e / NR) * a.ld + a.r0 + e % NR] = sum;
    }
    if (inext < Vc) finish(inext, xnext);
    consumer_sync(nct);
  }
}

// ------------------------------------------------------------------ coarse operator, FP32 vectors
// One pass over D_c for nrhs = 1 .. 4, 8, 12 or 16 right-hand sides (FP32 or FP16-scaled storage);
// the column-chunked apply_tma_kernel (kept for FP64 and other column counts) streams D_c once per
// 4 columns and stages the neighbour vectors in a separate per-site gather.  The stage of chunk (i, d)
// holds the stencil block (column-major, as in apply_tma_kernel) and the FP32 rows of x_c(nbr(i, d))
// (nc x NR values, contiguous in the coarse vector), both by bulk copy.  Consumer thread
// (cg, qg, rg) keeps rows rg*CPL .. rg*CPL + CPL - 1 and right-hand sides RW qg .. RW qg + RW - 1
// (RW = min(4, nrhs)) in registers and walks the stencil-block columns b = cg, cg + G, ...; per
// site a shared-memory sum
// over the G column groups.  The FGMRES extras: xscale[r] multiplies column r as it is read (the
// FP16 block scale too), and the scaled own rows (d = 0) go to vout.
template <typename LT, int NR>
struct MrhsArgs {
  const LT* D;
  const float* dscale;
  const int* nbr;
  const float2* x;
  float2* y;
  float2* vout;
  const double* xscale;
  const int* skip;
  unsigned* err;
  Geom g;
  int ns, G;
};

template <typename LT, int NR, int LPR>
__global__ void __launch_bounds__(288) apply_mrhs_kernel(const MrhsArgs<LT, NR> a) {
  constexpr int CPL = Vec16<LT>::CPL;
  constexpr int ROWS = CPL * LPR;  // rows per thread: LPR 16-byte loads of a block column
  constexpr int RW = NR < 4 ? NR : 4;  // right-hand sides per thread
  constexpr int QG = NR / RW;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int nc = a.g.nc, ns = a.ns;
  const long long nc2 = (long long)nc * nc;
  const unsigned dbytes = (unsigned)(nc2 * sizeof(LT)), xbytes = (unsigned)(nc * NR * sizeof(float2));
  const unsigned chunk = dbytes + xbytes;
  unsigned char* stages = sm + kPipeBytes;
  float2* red = reinterpret_cast<float2*>(stages + (size_t)ns * chunk);  // [G][NR][nc + 1]
  const int ncw = (blockDim.x - 32) >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&pp->full[s], 1);
      mbar_init(&pp->empty[s], ncw);
    }
    pp->abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const long long Vc = a.g.Vc;
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      long long c = 0;
      int s = 0;
      unsigned ph = 0;
      int nb[9], nx[9];
      const uint64_t pol = l2_evict_first_policy();  // D_c is streamed once per application
      if (blockIdx.x < Vc)
        for (int d = 0; d < 9; ++d) nx[d] = __ldg(a.nbr + blockIdx.x * 9LL + d);
      for (long long i = blockIdx.x; i < Vc && !pp->abort; i += gridDim.x) {
#pragma unroll
        for (int d = 0; d < 9; ++d) nb[d] = nx[d];
        if (i + gridDim.x < Vc)
#pragma unroll
          for (int d = 0; d < 9; ++d) nx[d] = __ldg(a.nbr + (i + gridDim.x) * 9 + d);
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 9; ++d) {
          if (c >= ns && !wait_phase(&pp->empty[s], ph ^ 1u, pp)) {
            abort_cta(pp, a.err);
            ok = false;
            break;
          }
          mbar_expect_tx(&pp->full[s], chunk);
          unsigned char* st = stages + (size_t)s * chunk;
          bulk_load_hint(st, a.D + (i * 9 + d) * nc2, dbytes, &pp->full[s], pol);
          bulk_load(st + dbytes, a.x + (long long)nb[d] * nc * NR, xbytes, &pp->full[s]);
          ++c;
          if (++s == ns) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
      }
      drain(pp, c, ns);
    }
    return;
  }
  const int t = threadIdx.x - 32, nct = blockDim.x - 32;
  const int Gc = nc / ROWS, per = Gc * QG;
  const int cg = t / per, rem = t % per, rg = rem % Gc, qg = rem / Gc;
  const bool active = cg < a.G;
  float sc[RW];
#pragma unroll
  for (int u = 0; u < RW; ++u) sc[u] = a.xscale ? (float)a.xscale[RW * qg + u] : 1.f;
  int s = 0;
  unsigned ph = 0;
  for (long long i = blockIdx.x; i < Vc; i += gridDim.x) {
    float2 acc[ROWS][RW];
#pragma unroll
    for (int q = 0; q < ROWS; ++q)
#pragma unroll
      for (int u = 0; u < RW; ++u) acc[q][u] = make_float2(0.f, 0.f);
    for (int d = 0; d < 9; ++d) {
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], ph, pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      const unsigned char* st = stages + (size_t)s * chunk;
      const float2* Xs = reinterpret_cast<const float2*>(st + dbytes);
      if (ok && active) {
        const LT* blk = reinterpret_cast<const LT*>(st) + rg * ROWS;
        const float f = a.dscale ? a.dscale[i * 9 + d] : 1.f;
        float fs[RW];
#pragma unroll
        for (int u = 0; u < RW; ++u) fs[u] = f * sc[u];
#pragma unroll 2
        for (int b = cg; b < nc; b += a.G) {
          float2 v[ROWS];
#pragma unroll
          for (int l = 0; l < LPR; ++l) {
            float2 vl[CPL];
            Vec16<LT>::ld(blk + (size_t)b * nc + l * CPL, vl);
#pragma unroll
            for (int q = 0; q < CPL; ++q) v[l * CPL + q] = vl[q];
          }
          float2 xv[RW];
          if constexpr (RW == 4) {
            const float4 x01 = *reinterpret_cast<const float4*>(Xs + b * NR + 4 * qg);
            const float4 x23 = *reinterpret_cast<const float4*>(Xs + b * NR + 4 * qg + 2);
            xv[0] = make_float2(x01.x, x01.y);
            xv[1] = make_float2(x01.z, x01.w);
            xv[2] = make_float2(x23.x, x23.y);
            xv[3] = make_float2(x23.z, x23.w);
          } else {
#pragma unroll
            for (int u = 0; u < RW; ++u) xv[u] = Xs[b * NR + RW * qg + u];
          }
#pragma unroll
          for (int u = 0; u < RW; ++u) xv[u] = make_float2(xv[u].x * fs[u], xv[u].y * fs[u]);
#pragma unroll
          for (int q = 0; q < ROWS; ++q)
#pragma unroll
            for (int u = 0; u < RW; ++u) cfma(acc[q][u], v[q], xv[u]);
        }
      }
      if (d == 0 && a.vout && ok)  // the own rows, scaled, for the Krylov basis
        for (int e = t; e < nc * NR; e += nct) {
          const float2 v = Xs[e];
          const float f = a.xscale ? (float)a.xscale[e % NR] : 1.f;
          a.vout[i * nc * NR + e] = make_float2(v.x * f, v.y * f);
        }
      __syncwarp();
      if ((t & 31) == 0) mbar_arrive(&pp->empty[s]);
      if (++s == ns) {
        s = 0;
        ph ^= 1u;
      }
    }
    if (active)
#pragma unroll
      for (int q = 0; q < ROWS; ++q)
#pragma unroll
        for (int u = 0; u < RW; ++u) red[((size_t)cg * NR + RW * qg + u) * (nc + 1) + rg * ROWS + q] = acc[q][u];
    consumer_sync(nct);
    for (int e = t; e < nc * NR; e += nct) {
      const int row = e / NR, col = e % NR;
      float2 sum = make_float2(0.f, 0.f);
      for (int gg = 0; gg < a.G; ++gg) {
        const float2 v = red[((size_t)gg * NR + col) * (nc + 1) + row];
        sum.x += v.x;
        sum.y += v.y;
      }
      a.y[i * nc * NR + e] = sum;
    }
    consumer_sync(nct);
  }
}

// ------------------------------------------------------------------ even/odd coarse operator
// The pieces of the even/odd-reduced coarse system (Schur complement on the even sites).  Items
// are the Vc/2 sites of one checkerboard parity in half-index order (site = site_of[h]; a
// neighbour j of the other parity is entry j / 2 of its half vector).  Item h streams chunks
// d = d0 .. d1 - 1: d = 0 the site's self block, or with inv0 its inverse (stored
// [Vc/2][nc col][nc row] by half index); d >= 1 the hop block D_c[site][d].  Chunk d multiplies
//   d = 0:  s0[h]                    (times xscale[r] when sc0; the scaled s0[h] goes to vout)
//   d >= 1: c1 * s1[nbr(site, d) / 2] (times xscale[r] when sc1)
// and y[h] = sum + delta vadd[h] (vadd optional).  With post_inv (and d0 = 1) one more chunk
// follows the hops: the inverse self block, applied to that sum (reduced in shared memory), so
// y[h] = D_ii^-1 (sum + delta vadd[h]).  Same pipeline as apply_tma_kernel.
template <typename LT, int NR>
struct EoArgs {
  using AT = typename Acc<LT>::type;
  const LT* D;
  const LT* Dinv;
  const int* nbr;
  const int* site_of;
  const AT* s0;
  const AT* s1;
  const AT* vadd;
  AT* y;
  AT* vout;
  const double* xscale;
  const int* skip;
  unsigned* err;
  Geom g;
  int ld, r0, ns, G, d0, d1, inv0, sc0, sc1, post_inv;
  double c1, delta;
};

template <typename LT, int NR>
__global__ void __launch_bounds__(288) eo_apply_kernel(const EoArgs<LT, NR> a) {
  using AT = typename Acc<LT>::type;
  constexpr int CPL = Vec16<LT>::CPL;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int nc = a.g.nc, K = 9 * nc, ns = a.ns;
  const long long nc2 = (long long)nc * nc;
  const unsigned chunk = (unsigned)(nc2 * sizeof(LT));
  unsigned char* stages = sm + kPipeBytes;
  AT* xs = reinterpret_cast<AT*>(stages + (size_t)ns * chunk);  // [2][K][NR]
  AT* red = xs + (size_t)2 * K * NR;
  const int ncw = (blockDim.x - 32) >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&pp->full[s], 1);
      mbar_init(&pp->empty[s], ncw);
    }
    pp->abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const long long Vh = a.g.Vc / 2;
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      long long c = 0;
      const int dend = a.d1 + (a.post_inv ? 1 : 0);  // chunk d1: the inverse self block
      for (long long h = blockIdx.x; h < Vh && !pp->abort; h += gridDim.x) {
        const long long site = __ldg(a.site_of + h);
        for (int d = a.d0; d < dend; ++d, ++c) {
          const int s = (int)(c % ns);
          const long long q = c / ns;
          if (c >= ns && !wait_phase(&pp->empty[s], (unsigned)((q - 1) & 1), pp)) {
            abort_cta(pp, a.err);
            break;
          }
          mbar_expect_tx(&pp->full[s], chunk);
          const LT* src = d == a.d1 ? a.Dinv + h * nc2
                                    : (d == 0 ? (a.inv0 ? a.Dinv + h * nc2 : a.D + site * 9 * nc2)
                                              : a.D + (site * 9 + d) * nc2);
          bulk_load_hint(stages + (size_t)s * chunk, src, chunk, &pp->full[s], l2_evict_first_policy());
        }
      }
      drain(pp, c, ns);
    }
    return;
  }
  const int t = threadIdx.x - 32, nct = blockDim.x - 32;
  const int Gc = nc / CPL, rc = t % Gc, grp = t / Gc;
  const AT c1 = AT{(decltype(AT{}.x))a.c1, 0};
  auto gather = [&](long long h, AT* buf) {
    const long long site = __ldg(a.site_of + h);
    for (int e = t; e < K * NR; e += nct) {
      const int k = e / NR, r = e % NR, d = k / nc, b = k % nc;
      if (d < a.d0 || d >= a.d1) continue;
      const AT* src = d == 0 ? a.s0 + (h * nc + b) * a.ld + a.r0 + r
                             : a.s1 + ((long long)(__ldg(a.nbr + site * 9 + d) >> 1) * nc + b) * a.ld + a.r0 + r;
      cp_async_elem(buf + e, src);
    }
    cp_async_commit();
  };
  auto finish = [&](long long h, AT* buf) {
    cp_async_wait_all();
    for (int e = t; e < K * NR; e += nct) {
      const int k = e / NR, r = e % NR, d = k / nc, b = k % nc;
      if (d < a.d0 || d >= a.d1) continue;
      AT v = buf[e];
      if (d == 0) {
        if (a.sc0) v = scaled(v, a.xscale[a.r0 + r]);
        if (a.vout) a.vout[(h * nc + b) * a.ld + a.r0 + r] = v;
      } else {
        if (a.sc1) v = scaled(v, a.xscale[a.r0 + r]);
        v = AT{v.x * c1.x, v.y * c1.x};
      }
      buf[e] = v;
    }
  };
  long long c = 0;
  int it = 0;
  if (blockIdx.x < Vh) {
    gather(blockIdx.x, xs);
    finish(blockIdx.x, xs);
  }
  consumer_sync(nct);
  for (long long h = blockIdx.x; h < Vh; h += gridDim.x, ++it) {
    AT* xcur = xs + (size_t)(it & 1) * K * NR;
    AT* xnext = xs + (size_t)((it + 1) & 1) * K * NR;
    const long long hnext = h + gridDim.x;
    if (hnext < Vh) gather(hnext, xnext);
    AT acc[CPL][NR];
    // one chunk: acc += block(chunk c) * X[xd]
    auto consume = [&](const AT* xd) {
      const int s = (int)(c % ns);
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], (unsigned)((c / ns) & 1), pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      if (ok && grp < a.G) {
        const LT* blk = reinterpret_cast<const LT*>(stages + (size_t)s * chunk) + rc * CPL;
#pragma unroll 4
        for (int b = grp; b < nc; b += a.G) {
          AT v[CPL];
          Vec16<LT>::ld(blk + (size_t)b * nc, v);
#pragma unroll
          for (int q = 0; q < CPL; ++q)
#pragma unroll
            for (int r = 0; r < NR; ++r) cfma(acc[q][r], v[q], xd[b * NR + r]);
        }
      }
      __syncwarp();
      if ((t & 31) == 0) mbar_arrive(&pp->empty[s]);
      ++c;
    };
    // sum over the column groups into out[nc][NR] (+ delta vadd[h])
    auto reduce_to = [&](AT* out, long long h, bool add) {
      if (grp < a.G)
#pragma unroll
        for (int q = 0; q < CPL; ++q)
#pragma unroll
          for (int r = 0; r < NR; ++r) red[((size_t)grp * nc + rc * CPL + q) * NR + r] = acc[q][r];
      consumer_sync(nct);
      for (int e = t; e < nc * NR; e += nct) {
        AT sum = AT{0, 0};
        for (int gg = 0; gg < a.G; ++gg) {
          const AT v = red[(size_t)gg * nc * NR + e];
          sum.x += v.x;
          sum.y += v.y;
        }
        const long long o = (h * nc + e / NR) * a.ld + a.r0 + e % NR;
        if (add && a.vadd) {
          const AT w = a.vadd[o];
          sum.x += (decltype(sum.x))a.delta * w.x;
          sum.y += (decltype(sum.x))a.delta * w.y;
        }
        if (out) out[e] = sum;
        else a.y[o] = sum;
      }
    };
    auto zero_acc = [&]() {
#pragma unroll
      for (int q = 0; q < CPL; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[q][r] = AT{0, 0};
    };
    zero_acc();
    for (int d = a.d0; d < a.d1; ++d) consume(xcur + (size_t)d * nc * NR);
    if (a.post_inv) {
      // z = sum (+ delta vadd) into the (unused) direction-0 slot, then y = D_ii^-1 z
      reduce_to(xcur, h, true);
      consumer_sync(nct);
      zero_acc();
      consume(xcur);
      reduce_to(nullptr, h, false);
    } else {
      reduce_to(nullptr, h, true);
    }
    if (hnext < Vh) finish(hnext, xnext);
    consumer_sync(nct);
  }
}

// The even/odd pieces for FP32 storage in the one-pass form of apply_mrhs_kernel: each stage holds
// one block (hop block, self block or stored inverse) and, for a hop or the self block, the
// source rows (s1 rows of the neighbour's half index, or the own s0 rows), both by bulk copy.
// Meaning of the arguments as for eo_apply_kernel (EoArgs).  With post_inv the hop sum (plus
// delta vadd) is reduced into shared memory and multiplied by the inverse block that the
// producer streams after the hops.
template <int NR>
__global__ void __launch_bounds__(288) eo_mrhs_kernel(const EoArgs<float2, NR> a) {
  constexpr int CPL = 2;
  constexpr int RW = NR < 4 ? NR : 4;
  constexpr int QG = NR / RW;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int nc = a.g.nc, ns = a.ns;
  const long long nc2 = (long long)nc * nc;
  const unsigned dbytes = (unsigned)(nc2 * sizeof(float2)), xbytes = (unsigned)(nc * NR * sizeof(float2));
  const unsigned chunk = dbytes + xbytes;
  unsigned char* stages = sm + kPipeBytes;
  float2* red = reinterpret_cast<float2*>(stages + (size_t)ns * chunk);  // [G][NR][nc + 1]
  float2* zb = red + (size_t)a.G * NR * (nc + 1);                        // [nc][NR] hop sum (post_inv)
  const int ncw = (blockDim.x - 32) >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&pp->full[s], 1);
      mbar_init(&pp->empty[s], ncw);
    }
    pp->abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const long long Vh = a.g.Vc / 2;
  const int dend = a.d1 + (a.post_inv ? 1 : 0);  // chunk d1 (post_inv): the inverse block
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      long long c = 0;
      int s = 0;
      unsigned ph = 0;
      for (long long h = blockIdx.x; h < Vh && !pp->abort; h += gridDim.x) {
        const long long site = __ldg(a.site_of + h);
        bool ok = true;
        for (int d = a.d0; d < dend; ++d) {
          if (c >= ns && !wait_phase(&pp->empty[s], ph ^ 1u, pp)) {
            abort_cta(pp, a.err);
            ok = false;
            break;
          }
          const bool post = d == a.d1;
          mbar_expect_tx(&pp->full[s], post ? dbytes : chunk);
          unsigned char* st = stages + (size_t)s * chunk;
          const float2* blk = post ? a.Dinv + h * nc2
                                   : (d == 0 ? (a.inv0 ? a.Dinv + h * nc2 : a.D + site * 9 * nc2)
                                             : a.D + (site * 9 + d) * nc2);
          bulk_load_hint(st, blk, dbytes, &pp->full[s], l2_evict_first_policy());
          if (!post) {
            const float2* src = d == 0 ? a.s0 + h * nc * NR
                                       : a.s1 + (long long)(__ldg(a.nbr + site * 9 + d) >> 1) * nc * NR;
            bulk_load(st + dbytes, src, xbytes, &pp->full[s]);
          }
          ++c;
          if (++s == ns) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
      }
      drain(pp, c, ns);
    }
    return;
  }
  const int t = threadIdx.x - 32, nct = blockDim.x - 32;
  const int Gc = nc / CPL, per = Gc * QG;
  const int cg = t / per, rem = t % per, rg = rem % Gc, qg = rem / Gc;
  const bool active = cg < a.G;
  float sx[RW];
#pragma unroll
  for (int u = 0; u < RW; ++u) sx[u] = a.xscale ? (float)a.xscale[RW * qg + u] : 1.f;
  int s = 0;
  unsigned ph = 0;
  for (long long h = blockIdx.x; h < Vh; h += gridDim.x) {
    float2 acc[CPL][RW];
    auto zero = [&]() {
#pragma unroll
      for (int q = 0; q < CPL; ++q)
#pragma unroll
        for (int u = 0; u < RW; ++u) acc[q][u] = make_float2(0.f, 0.f);
    };
    // one chunk with source rows X (nc x NR) scaled per column by fs
    auto consume = [&](const float2* X, const float (&fs)[RW], bool own) {
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], ph, pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      const unsigned char* st = stages + (size_t)s * chunk;
      const float2* Xs = X ? X : reinterpret_cast<const float2*>(st + dbytes);
      if (ok && active) {
        const float2* blk = reinterpret_cast<const float2*>(st) + rg * CPL;
#pragma unroll 2
        for (int b = cg; b < nc; b += a.G) {
          float2 v[CPL];
          Vec16<float2>::ld(blk + (size_t)b * nc, v);
          float2 xv[RW];
#pragma unroll
          for (int u = 0; u < RW; ++u) {
            const float2 x = Xs[b * NR + RW * qg + u];
            xv[u] = make_float2(x.x * fs[u], x.y * fs[u]);
          }
#pragma unroll
          for (int q = 0; q < CPL; ++q)
#pragma unroll
            for (int u = 0; u < RW; ++u) cfma(acc[q][u], v[q], xv[u]);
        }
      }
      if (own && a.vout && ok)  // the own rows, scaled, for the Krylov basis
        for (int e = t; e < nc * NR; e += nct) {
          const float2 v = Xs[e];
          const float f = a.xscale ? (float)a.xscale[e % NR] : 1.f;
          a.vout[h * nc * NR + e] = make_float2(v.x * f, v.y * f);
        }
      __syncwarp();
      if ((t & 31) == 0) mbar_arrive(&pp->empty[s]);
      if (++s == ns) {
        s = 0;
        ph ^= 1u;
      }
    };
    // sum over column groups into out [nc][NR] (shared) or y (+ delta vadd when add)
    auto reduce_to = [&](float2* out, bool add) {
      if (active)
#pragma unroll
        for (int q = 0; q < CPL; ++q)
#pragma unroll
          for (int u = 0; u < RW; ++u) red[((size_t)cg * NR + RW * qg + u) * (nc + 1) + rg * CPL + q] = acc[q][u];
      consumer_sync(nct);
      for (int e = t; e < nc * NR; e += nct) {
        const int row = e / NR, col = e % NR;
        float2 sum = make_float2(0.f, 0.f);
        for (int gg = 0; gg < a.G; ++gg) {
          const float2 v = red[((size_t)gg * NR + col) * (nc + 1) + row];
          sum.x += v.x;
          sum.y += v.y;
        }
        const long long o = h * nc * NR + e;
        if (add && a.vadd) {
          const float2 w = a.vadd[o];
          sum.x += (float)a.delta * w.x;
          sum.y += (float)a.delta * w.y;
        }
        if (out) out[e] = sum;
        else a.y[o] = sum;
      }
      consumer_sync(nct);
    };
    zero();
    for (int d = a.d0; d < a.d1; ++d) {
      float fs[RW];
#pragma unroll
      for (int u = 0; u < RW; ++u) {
        const float base = d == 0 ? 1.f : (float)a.c1;
        fs[u] = ((d == 0 ? a.sc0 : a.sc1) ? sx[u] : 1.f) * base;
      }
      consume(nullptr, fs, d == 0);
    }
    if (a.post_inv) {
      reduce_to(zb, true);
      zero();
      float one[RW];
#pragma unroll
      for (int u = 0; u < RW; ++u) one[u] = 1.f;
      consume(zb, one, false);
      reduce_to(nullptr, false);
    } else {
      reduce_to(nullptr, true);
    }
  }
}

// ------------------------------------------------------------------ restriction
// One CTA per block, launched in block order, so the CTAs resident at any time read neighbouring
// blocks.  y on the block is staged as ys[h][n][r]; warp w computes rows (h, j) of R_i^h y_i^h,
// the lanes striding over n with 16-byte streaming loads of the row and 16-byte shared loads of
// y, then a shuffle sum.  Many small CTAs (8 per SM) keep enough loads in flight.
template <typename ST, int NR>
__global__ void __launch_bounds__(256) restrict_kernel(const ST* __restrict__ R, const ST* __restrict__ y,
                                                       ST* __restrict__ yc, Geom g, int ld, int r0) {
  using AT = typename Acc<ST>::type;
  constexpr int CPL = Vec16<ST>::CPL;
  extern __shared__ __align__(16) unsigned char smraw[];
  AT* ys = reinterpret_cast<AT*>(smraw);
  const long long blk = blockIdx.x;
  const int nagg = g.nagg, ntv = g.ntv, Vb = (int)g.Vb;
  const long long origin = block_origin(g, blk);
  for (int e = threadIdx.x; e < Vb * 12 * NR; e += blockDim.x) {
    const int sl = e / (12 * NR), rem = e % (12 * NR), dof = rem / NR, r = rem % NR;
    const long long site = block_site_fast(g, origin, sl);
    const int hh = dof / 6, n = sl * 6 + dof % 6;
    ys[((size_t)hh * nagg + n) * NR + r] = y[(site * 12 + dof) * ld + r0 + r];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int row = warp; row < 2 * ntv; row += nw) {
    const int hh = row / ntv;
    const ST* Rrow = R + (blk * 2 * ntv + row) * (long long)nagg;
    const AT* yh = ys + (size_t)hh * nagg * NR;
    AT acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = AT{0, 0};
#pragma unroll 4
    for (int q = lane; q < nagg / CPL; q += 32) {
      AT v[CPL], yv[CPL * NR];
      Ld16<ST>::ld(Rrow + q * CPL, v);
      load_run<AT, CPL * NR>(yh + (size_t)q * CPL * NR, yv);
#pragma unroll
      for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int r = 0; r < NR; ++r) cfma(acc[r], v[k], yv[k * NR + r]);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const AT sum = warp_csum(acc[r]);
      if (lane == 0) yc[(blk * 2 * ntv + row) * ld + r0 + r] = sum;
    }
  }
}

// ------------------------------------------------------------------ prolongation
// Item = block; chunk = (h, n0): rows j = 0..ntv-1 of R_i^h restricted to n0 .. n0+nch-1, one bulk
// copy per row into stage [j][nch].  Consumer warp w owns stage w; lane l computes
// x[n] = sum_j conj(R[j][n]) x_c[h][j] for n = n0 + l, n0 + l + 32, ...
template <typename ST, int NR>
struct ProlongArgs {
  using AT = typename Acc<ST>::type;
  const ST* R;
  const ST* xc;
  ST* x;
  unsigned* err;
  Geom g;
  int ld, r0, nch;
};

template <typename ST, int NR>
__global__ void __launch_bounds__(160) prolong_tma_kernel(const ProlongArgs<ST, NR> a) {
  using AT = typename Acc<ST>::type;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int ncw = (blockDim.x - 32) >> 5, ns = ncw;
  const int nagg = a.g.nagg, ntv = a.g.ntv, nch = a.nch, cpa = nagg / nch;  // chunks per aggregate
  const unsigned rowb = (unsigned)(nch * sizeof(ST)), chunk = rowb * ntv;
  unsigned char* stages = sm + kPipeBytes;
  AT* xs = reinterpret_cast<AT*>(stages + (size_t)ns * chunk);  // [2][ntv][NR]
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&pp->full[s], 1);
      mbar_init(&pp->empty[s], 1);
    }
    pp->abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const long long nblk = a.g.Vc;
  if (threadIdx.x < 32) {
    long long c = 0;
    for (long long blk = blockIdx.x; blk < nblk && !pp->abort; blk += gridDim.x) {
      for (int k = 0; k < 2 * cpa; ++k, ++c) {
        const int s = (int)(c % ns);
        const long long q = c / ns;
        const int hh = k / cpa, n0 = (k % cpa) * nch;
        bool ok = true;
        if (threadIdx.x == 0) {
          if (c >= ns && !wait_phase(&pp->empty[s], (unsigned)((q - 1) & 1), pp)) {
            abort_cta(pp, a.err);
            ok = false;
          } else {
            mbar_expect_tx(&pp->full[s], chunk);
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        // lanes issue the ntv row copies; all complete on the stage's full barrier
        for (int j = threadIdx.x; j < ntv; j += 32)
          bulk_load_hint(stages + (size_t)s * chunk + (size_t)j * rowb,
                         a.R + ((blk * 2 + hh) * ntv + j) * (long long)nagg + n0, rowb, &pp->full[s],
                         l2_evict_first_policy());
        __syncwarp();
      }
    }
    if (threadIdx.x == 0) drain(pp, c, ns);
    return;
  }
  const int t = threadIdx.x - 32, nct = blockDim.x - 32, w = t >> 5, lane = t & 31;
  long long c = 0;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    consumer_sync(nct);
    for (int e = t; e < 2 * ntv * NR; e += nct) xs[e] = a.xc[(blk * 2 * ntv + e / NR) * a.ld + a.r0 + e % NR];
    consumer_sync(nct);
    for (int k = 0; k < 2 * cpa; ++k, ++c) {
      if ((int)(c % ncw) != w) continue;
      const int s = (int)(c % ns);
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], (unsigned)((c / ns) & 1), pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      const int hh = k / cpa, n0 = (k % cpa) * nch;
      const ST* st = reinterpret_cast<const ST*>(stages + (size_t)s * chunk);
      const AT* xh = xs + (size_t)hh * ntv * NR;
      const long long origin = block_origin(a.g, blk);
      for (int nl = lane; nl < nch; nl += 32) {
        AT acc[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = AT{0, 0};
        if (ok) {
#pragma unroll 4
          for (int j = 0; j < ntv; ++j) {
            const ST v = st[(size_t)j * nch + nl];
#pragma unroll
            for (int r = 0; r < NR; ++r) cfmac(acc[r], v, xh[j * NR + r]);
          }
        }
        const int n = n0 + nl, sl = n / 6, dof = hh * 6 + n % 6;
        const long long site = block_site_fast(a.g, origin, sl);
#pragma unroll
        for (int r = 0; r < NR; ++r) a.x[(site * 12 + dof) * a.ld + a.r0 + r] = acc[r];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pp->empty[s]);
    }
  }
}

// ------------------------------------------------------------------ launch helpers
template <typename K>
amg_status grid_for(const amg_coarse* h, K kernel, int threads, size_t smem, long long items, int* grid) {
  AMG_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
  if (per_sm < 1) return AMG_ERR_UNSUPPORTED;
  *grid = capped_grid(h, items, (long long)per_sm * amg_sm_count());
  return AMG_OK;
}

template <typename LT, int NR>
amg_status launch_apply_tma(amg_coarse* h, const LT* D, const float* dscale, const void* x, void* y, int ld, int r0,
                            cudaStream_t st, const int* skip, const double* xscale, void* vout) {
  using AT = typename Acc<LT>::type;
  constexpr int CPL = Vec16<LT>::CPL;
  const int nc = h->g.nc;
  if (nc % CPL) return AMG_ERR_UNSUPPORTED;
  const int threads = 288;
  const int Gc = nc / CPL;
  int G = (threads - 32) / Gc;
  if (G < 1) return AMG_ERR_UNSUPPORTED;
  if (G > nc) G = nc;
  const size_t chunk = (size_t)nc * nc * sizeof(LT);
  // three stages: a short ring lets more CTAs share an SM, which beats deeper prefetch here
  const int ns = 3;
  const size_t smem = kPipeBytes + ns * chunk + (size_t)2 * 9 * nc * NR * sizeof(AT) + (size_t)G * nc * NR * sizeof(AT);
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  int grid = 0;
  amg_status s = grid_for(h, apply_tma_kernel<LT, NR>, threads, smem, h->g.Vc, &grid);
  if (s != AMG_OK) return s;
  ApplyArgs<LT, NR> a{D, dscale, h->nbr, (const AT*)x, (AT*)y, (AT*)vout, xscale, skip, h->err, h->g, ld, r0, ns, G};
  apply_tma_kernel<LT, NR><<<grid, threads, smem, st>>>(a);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

template <typename LT, int NR, int LPR>
amg_status launch_apply_mrhs_rows(amg_coarse* h, const LT* D, const float* dscale, const void* x, void* y,
                                  cudaStream_t st, const int* skip, const double* xscale, void* vout) {
  constexpr int ROWS = Vec16<LT>::CPL * LPR;
  const int nc = h->g.nc;
  if (nc % ROWS) return AMG_ERR_UNSUPPORTED;
  const int per = (nc / ROWS) * (NR < 4 ? 1 : NR / 4);
  int G = 256 / per;
  if (G < 1) return AMG_ERR_UNSUPPORTED;
  if (G > nc) G = nc;
  const int threads = 32 + ((G * per + 31) / 32) * 32;
  const size_t chunk = (size_t)nc * nc * sizeof(LT) + (size_t)nc * NR * sizeof(float2);
  int ns = (int)((48 * 1024) / chunk);
  ns = ns < 2 ? 2 : (ns > 4 ? 4 : ns);
  const size_t smem = kPipeBytes + ns * chunk + (size_t)G * NR * (nc + 1) * sizeof(float2);
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  int grid = 0;
  amg_status s = grid_for(h, apply_mrhs_kernel<LT, NR, LPR>, threads, smem, h->g.Vc, &grid);
  if (s != AMG_OK) return s;
  MrhsArgs<LT, NR> a{D, dscale, h->nbr, (const float2*)x, (float2*)y, (float2*)vout, xscale, skip, h->err, h->g, ns, G};
  apply_mrhs_kernel<LT, NR, LPR><<<grid, threads, smem, st>>>(a);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

// FP32 storage with 4 or more columns: four rows per thread (two 16-byte loads of a block column)
// so that each thread's 16 complex products share 64 bytes of shared-memory loads.
template <typename LT, int NR>
amg_status launch_apply_mrhs(amg_coarse* h, const LT* D, const float* dscale, const void* x, void* y, cudaStream_t st,
                             const int* skip, const double* xscale, void* vout) {
  if constexpr (std::is_same<LT, float2>::value && NR >= 4) {
    if (h->g.nc % 4 == 0) return launch_apply_mrhs_rows<LT, NR, 2>(h, D, dscale, x, y, st, skip, xscale, vout);
  }
  return launch_apply_mrhs_rows<LT, NR, 1>(h, D, dscale, x, y, st, skip, xscale, vout);
}

struct EoCall {
  int parity, d0, d1, inv0, sc0, sc1, post_inv;
  const void *s0, *s1, *vadd;
  void *y, *vout;
  double c1, delta;
  const double* xscale;
  const int* skip;
};

template <int NR>
amg_status launch_eo_mrhs(amg_coarse* h, const EoCall& e, cudaStream_t st) {
  const int nc = h->g.nc;
  if (nc % 2) return AMG_ERR_UNSUPPORTED;
  const int per = (nc / 2) * (NR < 4 ? 1 : NR / 4);
  int G = 256 / per;
  if (G < 1) return AMG_ERR_UNSUPPORTED;
  if (G > nc) G = nc;
  const int threads = 32 + ((G * per + 31) / 32) * 32;
  const size_t chunk = (size_t)nc * nc * sizeof(float2) + (size_t)nc * NR * sizeof(float2);
  int ns = (int)((48 * 1024) / chunk);
  ns = ns < 2 ? 2 : (ns > 4 ? 4 : ns);
  const size_t smem =
      kPipeBytes + ns * chunk + (size_t)G * NR * (nc + 1) * sizeof(float2) + (size_t)nc * NR * sizeof(float2);
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  int grid = 0;
  amg_status s = grid_for(h, eo_mrhs_kernel<NR>, threads, smem, h->g.Vc / 2, &grid);
  if (s != AMG_OK) return s;
  EoArgs<float2, NR> a{(const float2*)h->Dq, (const float2*)h->Dinvq, h->nbr,
                       h->eo_site + (size_t)e.parity * (h->g.Vc / 2), (const float2*)e.s0, (const float2*)e.s1,
                       (const float2*)e.vadd, (float2*)e.y, (float2*)e.vout, e.xscale, e.skip, h->err, h->g, NR, 0, ns,
                       G, e.d0, e.d1, e.inv0, e.sc0, e.sc1, e.post_inv, e.c1, e.delta};
  eo_mrhs_kernel<NR><<<grid, threads, smem, st>>>(a);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

template <typename LT, int NR>
amg_status launch_eo(amg_coarse* h, const EoCall& e, int ld, int r0, cudaStream_t st) {
  using AT = typename Acc<LT>::type;
  constexpr int CPL = Vec16<LT>::CPL;
  const int nc = h->g.nc;
  if (nc % CPL) return AMG_ERR_UNSUPPORTED;
  const int threads = 288;
  const int Gc = nc / CPL;
  int G = (threads - 32) / Gc;
  if (G < 1) return AMG_ERR_UNSUPPORTED;
  if (G > nc) G = nc;
  const size_t chunk = (size_t)nc * nc * sizeof(LT);
  const int ns = 3;
  const size_t smem = kPipeBytes + ns * chunk + (size_t)2 * 9 * nc * NR * sizeof(AT) + (size_t)G * nc * NR * sizeof(AT);
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  int grid = 0;
  amg_status s = grid_for(h, eo_apply_kernel<LT, NR>, threads, smem, h->g.Vc / 2, &grid);
  if (s != AMG_OK) return s;
  EoArgs<LT, NR> a{(const LT*)h->Dq, (const LT*)h->Dinvq, h->nbr, h->eo_site + (size_t)e.parity * (h->g.Vc / 2),
                   (const AT*)e.s0, (const AT*)e.s1, (const AT*)e.vadd, (AT*)e.y, (AT*)e.vout, e.xscale, e.skip,
                   h->err, h->g, ld, r0, ns, G, e.d0, e.d1, e.inv0, e.sc0, e.sc1, e.post_inv, e.c1, e.delta};
  eo_apply_kernel<LT, NR><<<grid, threads, smem, st>>>(a);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

template <typename ST, int NR>
amg_status launch_restrict(amg_coarse* h, const ST* R, const ST* y, ST* yc, int ld, int r0, cudaStream_t st) {
  using AT = typename Acc<ST>::type;
  const size_t smem = (size_t)2 * h->g.nagg * NR * sizeof(AT);
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  if (smem > 48 * 1024)
    AMG_CUDA_TRY(cudaFuncSetAttribute(restrict_kernel<ST, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  restrict_kernel<ST, NR><<<(unsigned)h->g.Vc, 256, smem, st>>>(R, y, yc, h->g, ld, r0);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

// Largest nch dividing 6 Vb, a multiple of 6 (whole sites), with ntv * nch * sizeof(ST) <= 24 KB.
// Prolongation for FP32 R (one pass for nrhs <= 4 columns): one CTA per block, like the
// restriction.  R is stored row-major per test vector ([block][2 Ntv rows][nagg dofs]), so the
// output dofs read R by column: a thread owns two consecutive dofs n, n + 1 of one chirality half
// (the same site: a site has 6 dofs per half) and reads their 16 bytes of every row j < Ntv, a warp
// covering 512 contiguous bytes per row; x_c of the block sits in shared memory.  The rows are
// read with the streaming hint (read once) and x is written with one 16-byte streaming store per
// pair (1 RHS).  Measured 93 % of the copy bandwidth against 90 % for the bulk-copy ring form
// (prolong_tma_kernel, kept for FP64), whose single-dof lanes stored 8 bytes each.
template <int NR>
__global__ void __launch_bounds__(256) prolong_pair_kernel(const float2* __restrict__ R, const float2* __restrict__ xc,
                                                           float2* __restrict__ x, Geom g, int ld, int r0) {
  __shared__ float2 xs[2 * AMG_MAX_NTV * NR];
  const long long blk = blockIdx.x;
  const int nagg = g.nagg, ntv = g.ntv, npair = nagg / 2;
  for (int e = threadIdx.x; e < 2 * ntv * NR; e += blockDim.x) xs[e] = xc[(blk * 2 * ntv + e / NR) * ld + r0 + e % NR];
  __syncthreads();
  const long long origin = block_origin(g, blk);
  for (int p = threadIdx.x; p < 2 * npair; p += blockDim.x) {
    const int hh = p / npair, q = p % npair;
    const float2* Rp = R + ((blk * 2 + hh) * ntv) * (long long)nagg + 2 * q;
    const float2* xh = xs + (size_t)hh * ntv * NR;
    float2 a0[NR], a1[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) a0[r] = a1[r] = make_float2(0.f, 0.f);
#pragma unroll 5
    for (int j = 0; j < ntv; ++j) {
      const float4 v = __ldcs(reinterpret_cast<const float4*>(Rp + (size_t)j * nagg));
      const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        cfmac(a0[r], v0, xh[j * NR + r]);
        cfmac(a1[r], v1, xh[j * NR + r]);
      }
    }
    const int n = 2 * q, sl = n / 6, dof = hh * 6 + n % 6;
    float2* xo = x + (block_site_fast(g, origin, sl) * 12 + dof) * ld + r0;
    if (NR == 1 && ld == 1) {
      __stcs(reinterpret_cast<float4*>(xo), make_float4(a0[0].x, a0[0].y, a1[0].x, a1[0].y));
    } else {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        xo[r] = a0[r];
        xo[ld + r] = a1[r];
      }
    }
  }
}

template <typename ST>
int prolong_chunk(const Geom& g) {
  int best = 0;
  for (int nch = 6; nch <= g.nagg; nch += 6)
    if (g.nagg % nch == 0 && (size_t)g.ntv * nch * sizeof(ST) <= 24 * 1024 && (nch * sizeof(ST)) % 16 == 0)
      best = nch;
  return best;
}

template <int NR>
amg_status launch_prolong_pair(amg_coarse* h, const float2* R, const float2* xc, float2* x, int ld, int r0,
                               cudaStream_t st) {
  prolong_pair_kernel<NR><<<(unsigned)h->g.Vc, 256, 0, st>>>(R, xc, x, h->g, ld, r0);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

template <typename ST, int NR>
amg_status launch_prolong_tma(amg_coarse* h, const ST* R, const ST* xc, ST* x, int ld, int r0, cudaStream_t st) {
  using AT = typename Acc<ST>::type;
  const int threads = 32 + 4 * 32;
  const int ns = (threads - 32) / 32;  // one stage per consumer warp: the kernel derives it the same way
  const int nch = prolong_chunk<ST>(h->g);
  if (nch == 0) return AMG_ERR_UNSUPPORTED;
  const size_t chunk = (size_t)h->g.ntv * nch * sizeof(ST);
  const size_t smem = kPipeBytes + ns * chunk + (size_t)2 * h->g.ntv * NR * sizeof(AT);
  int grid = 0;
  amg_status s = grid_for(h, prolong_tma_kernel<ST, NR>, threads, smem, h->g.Vc, &grid);
  if (s != AMG_OK) return s;
  ProlongArgs<ST, NR> a{R, xc, x, h->err, h->g, ld, r0, nch};
  prolong_tma_kernel<ST, NR><<<grid, threads, smem, st>>>(a);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

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

template <typename LT>
amg_status apply_prec(amg_coarse* h, const LT* D, const float* dscale, const void* x, void* y, int nrhs,
                      cudaStream_t s, const int* skip, const double* xscale, void* vout) {
  if constexpr (!std::is_same<LT, double2>::value) {  // FP32 coarse vectors: one pass for these counts
    if (nrhs == 1) return launch_apply_mrhs<LT, 1>(h, D, dscale, x, y, s, skip, xscale, vout);
    if (nrhs == 2) return launch_apply_mrhs<LT, 2>(h, D, dscale, x, y, s, skip, xscale, vout);
    if (nrhs == 3) return launch_apply_mrhs<LT, 3>(h, D, dscale, x, y, s, skip, xscale, vout);
    if (nrhs == 4) return launch_apply_mrhs<LT, 4>(h, D, dscale, x, y, s, skip, xscale, vout);
    if (nrhs == 8) return launch_apply_mrhs<LT, 8>(h, D, dscale, x, y, s, skip, xscale, vout);
    if (nrhs == 12) return launch_apply_mrhs<LT, 12>(h, D, dscale, x, y, s, skip, xscale, vout);
    if (nrhs == 16) return launch_apply_mrhs<LT, 16>(h, D, dscale, x, y, s, skip, xscale, vout);
  }
  return for_rhs_chunks(nrhs, [&](int r0, int nr) {
    if (nr == 4) return launch_apply_tma<LT, 4>(h, D, dscale, x, y, nrhs, r0, s, skip, xscale, vout);
    if (nr == 2) return launch_apply_tma<LT, 2>(h, D, dscale, x, y, nrhs, r0, s, skip, xscale, vout);
    return launch_apply_tma<LT, 1>(h, D, dscale, x, y, nrhs, r0, s, skip, xscale, vout);
  });
}

}  // namespace

amg_status amg_internal_restrict(amg_coarse* h, const void* y, void* yc, int nrhs, cudaStream_t s) {
  if (h->p.vec_prec == AMG_BF16) return amg_internal_restrict_tc(h, y, yc, nrhs, s);
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
  if (h->p.vec_prec == AMG_BF16) return amg_internal_prolong_tc(h, xc, x, nrhs, s);
  if (h->p.vec_prec == AMG_FP64) {
    const double2* R = h->R64;
    return for_rhs_chunks(nrhs, [&](int r0, int nr) {
      if (nr == 4) return launch_prolong_tma<double2, 4>(h, R, (const double2*)xc, (double2*)x, nrhs, r0, s);
      if (nr == 2) return launch_prolong_tma<double2, 2>(h, R, (const double2*)xc, (double2*)x, nrhs, r0, s);
      return launch_prolong_tma<double2, 1>(h, R, (const double2*)xc, (double2*)x, nrhs, r0, s);
    });
  }
  if (h->p.vec_prec == AMG_FP32 && h->p.r_prec == AMG_FP32) {
    const float2* R = (const float2*)h->Rq;
    return for_rhs_chunks(nrhs, [&](int r0, int nr) {
      if (nr == 4) return launch_prolong_pair<4>(h, R, (const float2*)xc, (float2*)x, nrhs, r0, s);
      if (nr == 2) return launch_prolong_pair<2>(h, R, (const float2*)xc, (float2*)x, nrhs, r0, s);
      return launch_prolong_pair<1>(h, R, (const float2*)xc, (float2*)x, nrhs, r0, s);
    });
  }
  return AMG_ERR_UNSUPPORTED;
}

amg_status amg_internal_apply(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s) {
  return amg_internal_apply_ex(h, xc, yc, nrhs, s, nullptr, nullptr, nullptr);
}

amg_status amg_internal_apply_ex(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s,
                                 const int* skip, const double* xscale, void* vout) {
  switch (h->p.link_prec) {
    case AMG_FP64:
      if (h->p.vec_prec != AMG_FP64) return AMG_ERR_UNSUPPORTED;
      return apply_prec<double2>(h, (const double2*)h->Dq, nullptr, xc, yc, nrhs, s, skip, xscale, vout);
    case AMG_FP32:
      if (h->p.vec_prec == AMG_FP64) return AMG_ERR_UNSUPPORTED;
      // 4..16 columns: one pass on the tensor cores, tcgen05 with FP16 split operands up to nc = 56,
      // mma.sync with split-TF32 operands beyond (both measured faster than the one-pass SIMT kernel)
      if (h->tc5_x && nrhs >= 4 && nrhs <= 16) return amg_internal_apply_tc5(h, xc, yc, nrhs, s, skip, xscale, vout);
      if (h->Dtf && (nrhs == 4 || nrhs == 8 || nrhs == 12 || nrhs == 16))
        return amg_internal_apply_tf32(h, xc, yc, nrhs, s, skip, xscale, vout);
      return apply_prec<float2>(h, (const float2*)h->Dq, nullptr, xc, yc, nrhs, s, skip, xscale, vout);
    case AMG_FP16_SCALED:
      if (h->p.vec_prec == AMG_FP64) return AMG_ERR_UNSUPPORTED;
      if (h->tc5_x && nrhs >= 4 && nrhs <= 16) return amg_internal_apply_tc5(h, xc, yc, nrhs, s, skip, xscale, vout);
      return apply_prec<__half2>(h, (const __half2*)h->Dq, h->Dscale, xc, yc, nrhs, s, skip, xscale, vout);
    case AMG_BF16:
      return amg_internal_apply_tc(h, xc, yc, nrhs, s, skip, xscale, vout);
    default:
      return AMG_ERR_UNSUPPORTED;
  }
}

amg_status amg_internal_eo_apply(amg_coarse* h, int parity, int d0, int d1, bool inv0, const void* s0, bool sc0,
                                 const void* s1, double c1, bool sc1, const void* vadd, double delta, void* y,
                                 void* vout, const double* xscale, const int* skip, int nrhs, cudaStream_t st,
                                 bool post_inv) {
  if (!h->Dinvq || !h->eo_site) return AMG_ERR_UNSUPPORTED;
  if (post_inv && d0 == 0) return AMG_ERR_INVALID_ARG;  // the inverse takes the place of direction 0
  const EoCall e{parity, d0, d1, inv0 ? 1 : 0, sc0 ? 1 : 0, sc1 ? 1 : 0, post_inv ? 1 : 0,
                 s0, s1, vadd, y, vout, c1, delta, xscale, skip};
  if (h->p.link_prec == AMG_FP64 && h->p.vec_prec == AMG_FP64)
    return for_rhs_chunks(nrhs, [&](int r0, int nr) {
      if (nr == 4) return launch_eo<double2, 4>(h, e, nrhs, r0, st);
      if (nr == 2) return launch_eo<double2, 2>(h, e, nrhs, r0, st);
      return launch_eo<double2, 1>(h, e, nrhs, r0, st);
    });
  if (h->p.link_prec == AMG_FP32 && h->p.vec_prec != AMG_FP64) {
    switch (nrhs) {  // one pass: blocks and source rows through the ring
      case 1: return launch_eo_mrhs<1>(h, e, st);
      case 2: return launch_eo_mrhs<2>(h, e, st);
      case 3: return launch_eo_mrhs<3>(h, e, st);
      case 4: return launch_eo_mrhs<4>(h, e, st);
      case 8: return launch_eo_mrhs<8>(h, e, st);
      case 12: return launch_eo_mrhs<12>(h, e, st);
      case 16: return launch_eo_mrhs<16>(h, e, st);
      default: break;
    }
  }
  if (h->p.link_prec == AMG_FP32 && h->p.vec_prec != AMG_FP64)
    return for_rhs_chunks(nrhs, [&](int r0, int nr) {
      if (nr == 4) return launch_eo<float2, 4>(h, e, nrhs, r0, st);
      if (nr == 2) return launch_eo<float2, 2>(h, e, nrhs, r0, st);
      return launch_eo<float2, 1>(h, e, nrhs, r0, st);
    });
  return AMG_ERR_UNSUPPORTED;
}
