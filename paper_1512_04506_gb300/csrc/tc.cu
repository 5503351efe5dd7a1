// Multi-right-hand-side coarse operator on the tensor cores: y_c = D_c x_c for nrhs = 4, 8, 12 or 16
// right-hand sides with D_c stored as BF16 Re/Im planes and FP32 accumulation (the serving form of
// Alg. 2's coarse-operator application; Sec. 3 stores D_c in half precision).
//
// Complex products become one real product per stencil block d:
//     [Y_re | Y_im] += [A_re | A_im] . [[X_re, X_im], [-X_im, X_re]]
// with A = D_c[i][d] (nc x nc) and X = x_c(nbr(i, d)) (nc x nrhs), so M = nc, K = 2 nc and
// N = 2 nrhs.  The N axis is ordered in groups of 8 columns (Re of 4 right-hand sides, then Im of
// the same 4), so each 16x8 accumulator tile holds complete complex outputs.  A comes from the
// D_c stream (cp.async.bulk into an mbarrier ring, as in stream.cu); X is converted to BF16 once
// per call into padded BF16 planes (xc_to_planes_kernel), and the producer warp copies, next to
// each stencil block D_c[i][d], the planes of the neighbour nbr(i, d) into the same stage, so the
// consumers only issue tensor-core instructions.  Warp w of the consumers owns rows 16 w .. 16 w + 15
// of the site's output and all N columns.
#include "amg_internal.cuh"
#include "pipe.cuh"

namespace {
using namespace amgpipe;

typedef __nv_bfloat16 bf16;

__device__ inline void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ inline unsigned lds32(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }

struct TcApplyArgs {
  const bf16* D;   // [Vc][9][2][nc][nc]: Re plane then Im plane, row-major (row a, column b)
  const bf16* X;   // [Vc][xpitch]: the coarse vector in BF16 planes, see xc_to_planes_kernel
  const int* nbr;
  float2* y;
  const int* skip;
  unsigned* err;
  Geom g;
  int ns, xpitch;
};

// Coarse vector (FP32, [Vc][nc][nrhs], optionally times xscale[r]; the (scaled) FP32 vector is also
// stored to vout when given) -> BF16 planes per site: plane p (0 Re, 1 Im) at offset p * (nrhs (nc + 8) + 32),
// row r of length nc + 8 (8 pad); the paddings put the two planes and consecutive rows on
// different shared-memory banks once a site's block is copied to shared memory.
template <int NRHS>
__global__ void xc_to_planes_kernel(const float2* __restrict__ x, bf16* __restrict__ X, int nc, long long Vc,
                                    int xpitch, const double* __restrict__ xscale, float2* __restrict__ vout,
                                    const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int prow = nc + 8, pplane = NRHS * prow + 32;
  const long long total = Vc * nc * NRHS;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % NRHS);
    const long long ib = e / NRHS;
    const int b = (int)(ib % nc);
    const long long i = ib / nc;
    float2 v = x[e];
    if (xscale) {
      const float f = (float)xscale[r];
      v.x *= f;
      v.y *= f;
    }
    if (vout) vout[e] = v;
    bf16* site = X + i * xpitch;
    site[r * prow + b] = __float2bfloat16_rn(v.x);
    site[pplane + r * prow + b] = __float2bfloat16_rn(v.y);
  }
}

template <int NRHS>
__global__ void __launch_bounds__(160) apply_tc_kernel(const TcApplyArgs a) {
  constexpr int NT = NRHS / 4;  // n-tiles of 8 columns
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int nc = a.g.nc, ns = a.ns, mt_count = nc / 16;
  const unsigned dbytes = (unsigned)(2 * nc * nc * sizeof(bf16));
  const unsigned xbytes = (unsigned)(a.xpitch * sizeof(bf16));
  const unsigned chunk = dbytes + xbytes;  // stencil block d of D_c and the neighbour's planes
  unsigned char* stages = sm + kPipeBytes;
  const int xrow = nc + 8, xplane = NRHS * xrow + 32;
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
          unsigned char* st = stages + (size_t)s * chunk;
          bulk_load(st, a.D + (i * 9 + d) * 2LL * nc * nc, dbytes, &pp->full[s]);
          bulk_load(st + dbytes, a.X + (long long)a.nbr[i * 9 + d] * a.xpitch, xbytes, &pp->full[s]);
        }
      }
      drain(pp, c, ns);
    }
    return;
  }
  const int t = threadIdx.x - 32, w = t >> 5, lane = t & 31;
  const int g = lane >> 2, tq = lane & 3;
  long long c = 0;
  for (long long i = blockIdx.x; i < Vc; i += gridDim.x) {
    float acc[NT][4];
#pragma unroll
    for (int q = 0; q < NT; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[q][u] = 0.f;
    for (int d = 0; d < 9; ++d, ++c) {
      const int s = (int)(c % ns);
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], (unsigned)((c / ns) & 1), pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      if (ok && w < mt_count) {
        const bf16* Ablk = reinterpret_cast<const bf16*>(stages + (size_t)s * chunk);
        const bf16* xs = reinterpret_cast<const bf16*>(stages + (size_t)s * chunk + dbytes);
        const int row0 = w * 16 + g;
        for (int kk = 0; kk < 2 * (nc / 16); ++kk) {
          const int p = kk / (nc / 16), k0 = (kk % (nc / 16)) * 16;  // p = 0: A_re, 1: A_im
          const bf16* P = Ablk + (size_t)p * nc * nc;
          unsigned af[4];
          af[0] = lds32(P + (size_t)row0 * nc + k0 + 2 * tq);
          af[1] = lds32(P + (size_t)(row0 + 8) * nc + k0 + 2 * tq);
          af[2] = lds32(P + (size_t)row0 * nc + k0 + 8 + 2 * tq);
          af[3] = lds32(P + (size_t)(row0 + 8) * nc + k0 + 8 + 2 * tq);
#pragma unroll
          for (int q = 0; q < NT; ++q) {
            // column g of tile q: half = g / 4 (0: Re output, 1: Im output), rhs r = 4 q + g % 4
            const int half = g >> 2, r = 4 * q + (g & 3);
            const int sp = (p == half) ? 0 : 1;  // X_re or X_im
            const bf16* xb = xs + (size_t)sp * xplane + (size_t)r * xrow + k0 + 2 * tq;
            unsigned b0 = lds32(xb), b1 = lds32(xb + 8);
            if (p == 1 && half == 0) {
              b0 ^= 0x80008000u;
              b1 ^= 0x80008000u;
            }
            mma_bf16(acc[q], af, b0, b1);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pp->empty[s]);
    }
    // tile q, lane (g, tq): c0, c1 = rows g, cols 2 tq, 2 tq + 1; c2, c3 = row g + 8.
    // Columns 0..3 are Re of rhs 4q..4q+3, columns 4..7 their Im: lanes tq = 0, 1 hold Re and
    // receive the Im from lane tq + 2.
    if (w < mt_count) {
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        const float i0 = __shfl_down_sync(0xffffffffu, acc[q][0], 2);
        const float i1 = __shfl_down_sync(0xffffffffu, acc[q][1], 2);
        const float i2 = __shfl_down_sync(0xffffffffu, acc[q][2], 2);
        const float i3 = __shfl_down_sync(0xffffffffu, acc[q][3], 2);
        if (tq < 2) {
          const int r = 4 * q + 2 * tq;
          const int row = w * 16 + g;
          float4* y0 = reinterpret_cast<float4*>(a.y + (i * nc + row) * NRHS + r);
          float4* y1 = reinterpret_cast<float4*>(a.y + (i * nc + row + 8) * NRHS + r);
          *y0 = make_float4(acc[q][0], i0, acc[q][1], i1);
          *y1 = make_float4(acc[q][2], i2, acc[q][3], i3);
        }
      }
    }
  }
}

int sm_count_tc() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

// ------------------------------------------------------------------ R and P on the tensor cores
// R in BF16 planes, tiled for the tensor cores: Rtc[blk][c][h][p][j][48], chunk c covering the
// aggregate dofs n = 48 c .. 48 c + 47 (block-local sites 8 c .. 8 c + 7), p = 0 (Re), 1 (Im).
// Restriction:  [Yc_re | Yc_im] = [R_re | R_im] . [[Y_re, Y_im], [-Y_im, Y_re]]  (M = ntv, K = 2 n)
// Prolongation: [X_re | X_im] = [Q_re | Q_im] . [[c_re, c_im], [-c_im, c_re]]   (M = n, K = 2 ntv)
// with Q = R^dagger, Q_re = R_re^T, Q_im = -R_im^T.

__device__ inline void ldsm_x4_trans(unsigned (&r)[4], const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}

struct TcRPArgs {
  const bf16* R;       // Rtc
  const void* in;      // restrict: fine BF16 y; prolong: coarse FP32 x_c
  void* out;           // restrict: coarse FP32 y_c; prolong: fine BF16 x
  unsigned* err;
  Geom g;
  int ns, run;         // run = consecutive sites of a chunk that are consecutive on the lattice
};

// Block-local sites 8c .. 8c+7 as (8 / run) runs of `run` lattice-consecutive sites.
__device__ inline long long chunk_site(const Geom& g, long long blk, int c, int u, int run) {
  return block_site_fast(g, block_origin(g, blk), 8 * c + u * run);
}

template <int NRHS>
__global__ void __launch_bounds__(160) restrict_tc_kernel(const TcRPArgs a) {
  constexpr int NT = NRHS / 4;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int ntv = a.g.ntv, ns = a.ns, run = a.run, cpb = (int)(a.g.Vb / 8);  // chunks per block
  const int mts = (ntv + 15) / 16;                                          // m-tiles per chirality
  const unsigned rbytes = (unsigned)(2 * 2 * ntv * 48 * sizeof(bf16));
  const unsigned ybytes = (unsigned)(8 * 12 * NRHS * 4);
  const unsigned chunk = rbytes + ybytes + 1024;  // slack: padded A rows read past the last plane
  unsigned char* stages = sm + kPipeBytes;
  const int yrow = 48 + 8, yplane = 2 * NRHS * yrow + 32;  // Ybuf[buf][plane][h][r][n]
  bf16* ybuf = reinterpret_cast<bf16*>(stages + (size_t)ns * chunk);
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
  const long long nblk = a.g.Vc;
  const __nv_bfloat162* Y = reinterpret_cast<const __nv_bfloat162*>(a.in);
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      long long c = 0;
      for (long long blk = blockIdx.x; blk < nblk && !pp->abort; blk += gridDim.x) {
        for (int cc = 0; cc < cpb; ++cc, ++c) {
          const int s = (int)(c % ns);
          const long long q = c / ns;
          if (c >= ns && !wait_phase(&pp->empty[s], (unsigned)((q - 1) & 1), pp)) {
            abort_cta(pp, a.err);
            break;
          }
          mbar_expect_tx(&pp->full[s], rbytes + ybytes);
          unsigned char* st = stages + (size_t)s * chunk;
          bulk_load(st, a.R + (blk * cpb + cc) * (long long)(rbytes / sizeof(bf16)), rbytes, &pp->full[s]);
          const unsigned rb = (unsigned)(run * 12 * NRHS * 4);
          for (int u = 0; u < 8 / run; ++u) {
            const long long site = chunk_site(a.g, blk, cc, u, run);
            bulk_load(st + rbytes + u * rb, Y + site * 12 * NRHS, rb, &pp->full[s]);
          }
        }
      }
      drain(pp, c, ns);
    }
    return;
  }
  const int t = threadIdx.x - 32, nct = blockDim.x - 32, w = t >> 5, lane = t & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int hw = w / mts, mt = w % mts;  // warp -> (chirality, m-tile)
  long long c = 0;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    float acc[NT][4];
#pragma unroll
    for (int q = 0; q < NT; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[q][u] = 0.f;
    for (int cc = 0; cc < cpb; ++cc, ++c) {
      const int s = (int)(c % ns);
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], (unsigned)((c / ns) & 1), pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      const unsigned char* st = stages + (size_t)s * chunk;
      const __nv_bfloat162* Ys = reinterpret_cast<const __nv_bfloat162*>(st + rbytes);
      bf16* yb = ybuf + (size_t)(c & 1) * 2 * yplane;
      // Y of the chunk into planes yb[plane][h][r][n] (n = aggregate dof within the chunk)
      for (int e = t; e < 8 * 12 * NRHS && ok; e += nct) {
        const int r = e % NRHS, dofs = e / NRHS, sl = dofs / 12, dof = dofs % 12;
        const int h = dof / 6, n = sl * 6 + dof % 6;
        const __nv_bfloat162 v = Ys[e];
        yb[((size_t)h * NRHS + r) * yrow + n] = v.x;
        yb[yplane + ((size_t)h * NRHS + r) * yrow + n] = v.y;
      }
      consumer_sync(nct);
      if (ok && hw < 2) {
        const bf16* Rb = reinterpret_cast<const bf16*>(st);
        const int row0 = mt * 16 + g;
        for (int kk = 0; kk < 6; ++kk) {
          const int p = kk / 3, k0 = (kk % 3) * 16;  // p = 0: R_re, 1: R_im; k = n within the chunk
          const bf16* P = Rb + (size_t)((hw * 2 + p) * ntv) * 48;
          unsigned af[4];
          af[0] = lds32(P + (size_t)row0 * 48 + k0 + 2 * tq);
          af[1] = lds32(P + (size_t)(row0 + 8) * 48 + k0 + 2 * tq);
          af[2] = lds32(P + (size_t)row0 * 48 + k0 + 8 + 2 * tq);
          af[3] = lds32(P + (size_t)(row0 + 8) * 48 + k0 + 8 + 2 * tq);
#pragma unroll
          for (int q = 0; q < NT; ++q) {
            const int half = g >> 2, r = 4 * q + (g & 3);
            const int sp = (p == half) ? 0 : 1;
            const bf16* xb = yb + (size_t)sp * yplane + ((size_t)hw * NRHS + r) * yrow + k0 + 2 * tq;
            unsigned b0 = lds32(xb), b1 = lds32(xb + 8);
            if (p == 1 && half == 0) {
              b0 ^= 0x80008000u;
              b1 ^= 0x80008000u;
            }
            mma_bf16(acc[q], af, b0, b1);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pp->empty[s]);
    }
    // rows j = mt*16 + g (+8) < ntv of chirality hw: y_c[blk][hw][j][r]
    if (hw < 2) {
      float2* yc = reinterpret_cast<float2*>(a.out);
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        const float i0 = __shfl_down_sync(0xffffffffu, acc[q][0], 2);
        const float i1 = __shfl_down_sync(0xffffffffu, acc[q][1], 2);
        const float i2 = __shfl_down_sync(0xffffffffu, acc[q][2], 2);
        const float i3 = __shfl_down_sync(0xffffffffu, acc[q][3], 2);
        if (tq < 2) {
          const int r = 4 * q + 2 * tq, j0 = mt * 16 + g;
          if (j0 < ntv)
            *reinterpret_cast<float4*>(yc + ((blk * 2 + hw) * ntv + j0) * NRHS + r) =
                make_float4(acc[q][0], i0, acc[q][1], i1);
          if (j0 + 8 < ntv)
            *reinterpret_cast<float4*>(yc + ((blk * 2 + hw) * ntv + j0 + 8) * NRHS + r) =
                make_float4(acc[q][2], i2, acc[q][3], i3);
        }
      }
    }
  }
}

template <int NRHS>
__global__ void __launch_bounds__(224) prolong_tc_kernel(const TcRPArgs a) {
  constexpr int NT = NRHS / 4;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int ntv = a.g.ntv, ns = a.ns, run = a.run, cpb = (int)(a.g.Vb / 8);
  const unsigned chunk = (unsigned)(2 * 2 * ntv * 48 * sizeof(bf16));
  unsigned char* stages = sm + kPipeBytes;
  const int crow = ntv + 8, cplane = 2 * NRHS * crow + 32;  // cbuf[plane][h][r][j]
  bf16* cbuf = reinterpret_cast<bf16*>(stages + (size_t)ns * chunk);
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
  const long long nblk = a.g.Vc;
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      long long c = 0;
      for (long long blk = blockIdx.x; blk < nblk && !pp->abort; blk += gridDim.x) {
        for (int cc = 0; cc < cpb; ++cc, ++c) {
          const int s = (int)(c % ns);
          const long long q = c / ns;
          if (c >= ns && !wait_phase(&pp->empty[s], (unsigned)((q - 1) & 1), pp)) {
            abort_cta(pp, a.err);
            break;
          }
          mbar_expect_tx(&pp->full[s], chunk);
          bulk_load(stages + (size_t)s * chunk, a.R + (blk * cpb + cc) * (long long)(chunk / sizeof(bf16)), chunk,
                    &pp->full[s]);
        }
      }
      drain(pp, c, ns);
    }
    return;
  }
  const int t = threadIdx.x - 32, nct = blockDim.x - 32, w = t >> 5, lane = t & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int hw = w / 3, mt = w % 3;  // warp -> (chirality, m-tile of 16 dofs)
  const float2* xc = reinterpret_cast<const float2*>(a.in);
  __nv_bfloat162* X = reinterpret_cast<__nv_bfloat162*>(a.out);
  long long c = 0;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    consumer_sync(nct);
    for (int e = t; e < 2 * ntv * NRHS; e += nct) {
      const int r = e % NRHS, hj = e / NRHS, h = hj / ntv, j = hj % ntv;
      const float2 v = xc[(blk * 2 * ntv + hj) * NRHS + r];
      cbuf[((size_t)h * NRHS + r) * crow + j] = __float2bfloat16_rn(v.x);
      cbuf[cplane + ((size_t)h * NRHS + r) * crow + j] = __float2bfloat16_rn(v.y);
    }
    consumer_sync(nct);
    for (int cc = 0; cc < cpb; ++cc, ++c) {
      const int s = (int)(c % ns);
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], (unsigned)((c / ns) & 1), pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      if (ok && hw < 2) {
        const bf16* Rb = reinterpret_cast<const bf16*>(stages + (size_t)s * chunk);
        const long long origin = block_origin(a.g, blk);
        float acc[NT][4];
#pragma unroll
        for (int q = 0; q < NT; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[q][u] = 0.f;
        for (int k0 = 0; k0 < 2 * ntv; k0 += 16) {
          // A = [Q_re | Q_im] rows n = mt*16.., columns k = k0..k0+15: four transposed 8x8 tiles
          const int tile = lane >> 3, kt = k0 + (tile >> 1) * 8 + (lane & 7), n0 = mt * 16 + (tile & 1) * 8;
          const int pl = kt < ntv ? 0 : 1, j = kt < ntv ? kt : kt - ntv;
          unsigned af[4];
          ldsm_x4_trans(af, Rb + ((size_t)(hw * 2 + pl) * ntv + j) * 48 + n0);
          // Q_im = -R_im^T: negate the registers whose 8 k-columns lie in the R_im plane
          if (k0 >= ntv) {
            af[0] ^= 0x80008000u;
            af[1] ^= 0x80008000u;
          }
          if (k0 + 8 >= ntv) {
            af[2] ^= 0x80008000u;
            af[3] ^= 0x80008000u;
          }
#pragma unroll
          for (int q = 0; q < NT; ++q) {
            const int half = g >> 2, r = 4 * q + (g & 3);
            // B[k][col]: k < ntv (Q_re part): c_re (half 0) / c_im (half 1); k >= ntv: -c_im / c_re
            unsigned b[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int k = k0 + 8 * u + 2 * tq, p = k < ntv ? 0 : 1, jj = k < ntv ? k : k - ntv;
              const int sp = (p == half) ? 0 : 1;
              b[u] = lds32(cbuf + (size_t)sp * cplane + ((size_t)hw * NRHS + r) * crow + jj);
              if (p == 1 && half == 0) b[u] ^= 0x80008000u;
            }
            mma_bf16(acc[q], af, b[0], b[1]);
          }
        }
        // rows n = mt*16 + g (+8): aggregate dof of chirality hw within the chunk
#pragma unroll
        for (int q = 0; q < NT; ++q) {
          const float i0 = __shfl_down_sync(0xffffffffu, acc[q][0], 2);
          const float i1 = __shfl_down_sync(0xffffffffu, acc[q][1], 2);
          const float i2 = __shfl_down_sync(0xffffffffu, acc[q][2], 2);
          const float i3 = __shfl_down_sync(0xffffffffu, acc[q][3], 2);
          if (tq < 2) {
            const int r = 4 * q + 2 * tq;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int n = mt * 16 + g + 8 * u, sl = n / 6, dof = hw * 6 + n % 6;
              const long long site = block_site_fast(a.g, origin, 8 * cc + sl);
              __nv_bfloat162 v0 = __floats2bfloat162_rn(u ? acc[q][2] : acc[q][0], u ? i2 : i0);
              __nv_bfloat162 v1 = __floats2bfloat162_rn(u ? acc[q][3] : acc[q][1], u ? i3 : i1);
              uint2 pk;
              memcpy(&pk.x, &v0, 4);
              memcpy(&pk.y, &v1, 4);
              *reinterpret_cast<uint2*>(X + (site * 12 + dof) * NRHS + r) = pk;
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pp->empty[s]);
    }
  }
}

// R64 [blk][h][j][n] (complex double) -> Rtc [blk][c][h][p][j][48] (BF16, round to nearest even)
__global__ void r_to_tc_kernel(const double2* __restrict__ R, bf16* __restrict__ out, Geom g) {
  const int ntv = g.ntv, nagg = g.nagg, cpb = (int)(g.Vb / 8);
  const long long total = g.Vc * 2LL * ntv * nagg;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e % nagg);
    const long long q = e / nagg;
    const int j = (int)(q % ntv), h = (int)((q / ntv) % 2);
    const long long blk = q / (2LL * ntv);
    const int c = n / 48, nn = n % 48;
    const double2 v = R[e];
    const long long base = ((blk * cpb + c) * 2 + h) * 2;
    out[((base + 0) * ntv + j) * 48 + nn] = __double2bfloat16(v.x);
    out[((base + 1) * ntv + j) * 48 + nn] = __double2bfloat16(v.y);
  }
}

template <int NRHS, bool RESTRICT>
amg_status launch_rp_tc(amg_coarse* h, const void* in, void* out, cudaStream_t st) {
  const Geom& g = h->g;
  const int run = g.B[0] >= 8 ? 8 : g.B[0];
  const int mts = (g.ntv + 15) / 16;
  const int threads = RESTRICT ? 32 + 32 * 2 * mts : 32 + 32 * 6;
  size_t chunk, extra;
  if (RESTRICT) {
    chunk = (size_t)2 * 2 * g.ntv * 48 * sizeof(bf16) + 8 * 12 * NRHS * 4 + 1024;
    extra = (size_t)2 * 2 * (2 * NRHS * (48 + 8) + 32) * sizeof(bf16);
  } else {
    chunk = (size_t)2 * 2 * g.ntv * 48 * sizeof(bf16);
    extra = (size_t)2 * (2 * NRHS * (g.ntv + 8) + 32) * sizeof(bf16);
  }
  const int ns = 4;
  const size_t smem = kPipeBytes + ns * chunk + extra;
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  auto kern = RESTRICT ? restrict_tc_kernel<NRHS> : prolong_tc_kernel<NRHS>;
  AMG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  if (per_sm < 1) return AMG_ERR_UNSUPPORTED;
  const long long gmax = (long long)per_sm * sm_count_tc();
  const int grid = (int)(g.Vc < gmax ? g.Vc : gmax);
  TcRPArgs a{(const bf16*)h->Rtc, in, out, h->err, g, ns, run};
  kern<<<grid, threads, smem, st>>>(a);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

// D_c (canonical FP64 [Vc][9][nc][nc]) -> BF16 planes [Vc][9][2][nc][nc], round to nearest even.
__global__ void dc_to_bf16_kernel(const double2* __restrict__ Dc, bf16* __restrict__ out, int nc, long long nblk) {
  const long long n2 = (long long)nc * nc, total = nblk * n2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / n2, rem = e % n2;
    const double2 v = Dc[e];
    out[blk * 2 * n2 + rem] = __double2bfloat16(v.x);
    out[blk * 2 * n2 + n2 + rem] = __double2bfloat16(v.y);
  }
}

__global__ void bf16_to_dc_kernel(const bf16* __restrict__ in, double2* __restrict__ out, int nc, long long nblk) {
  const long long n2 = (long long)nc * nc, total = nblk * n2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / n2, rem = e % n2;
    out[e] = make_double2((double)__bfloat162float(in[blk * 2 * n2 + rem]),
                          (double)__bfloat162float(in[blk * 2 * n2 + n2 + rem]));
  }
}

int tc_xpitch(const Geom& g, int nrhs) { return ((2 * nrhs * (g.nc + 8) + 64) + 7) / 8 * 8; }

template <int NRHS>
amg_status launch_apply_tc(amg_coarse* h, const void* x, void* y, cudaStream_t st, const int* skip,
                           const double* xscale, void* vout) {
  const int nc = h->g.nc;
  const int xpitch = tc_xpitch(h->g, NRHS);
  if ((size_t)h->g.Vc * xpitch * sizeof(bf16) > h->tc_xbytes) return AMG_ERR_INVALID_ARG;  // nrhs > max_nrhs
  xc_to_planes_kernel<NRHS><<<4 * 152, 256, 0, st>>>((const float2*)x, (bf16*)h->tc_x, nc, h->g.Vc, xpitch, xscale,
                                                     (float2*)vout, skip);
  AMG_LAUNCH_CHECK();
  h->launches++;
  const int threads = 32 + 32 * (nc / 16);
  const size_t chunk = (size_t)2 * nc * nc * sizeof(bf16) + (size_t)xpitch * sizeof(bf16);
  int ns = (int)((72 * 1024) / chunk);
  ns = ns < 2 ? 2 : (ns > 6 ? 6 : ns);
  const size_t smem = kPipeBytes + ns * chunk;
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  AMG_CUDA_TRY(cudaFuncSetAttribute(apply_tc_kernel<NRHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_tc_kernel<NRHS>, threads, smem));
  if (per_sm < 1) return AMG_ERR_UNSUPPORTED;
  const long long gmax = (long long)per_sm * sm_count_tc();
  const int grid = (int)(h->g.Vc < gmax ? h->g.Vc : gmax);
  TcApplyArgs a{(const bf16*)h->Dtc, (const bf16*)h->tc_x, h->nbr, (float2*)y, skip, h->err, h->g, ns, xpitch};
  apply_tc_kernel<NRHS><<<grid, threads, smem, st>>>(a);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

}  // namespace

amg_status amg_internal_tc_prepare(amg_coarse* h, cudaStream_t st) {
  if (h->p.link_prec == AMG_BF16) {
    if (h->g.nc % 16 || h->g.nc > 64) return AMG_ERR_UNSUPPORTED;
    const size_t n = (size_t)h->g.Vc * 9 * 2 * h->g.nc * h->g.nc;
    AMG_CUDA_TRY(cudaMalloc(&h->Dtc, n * sizeof(bf16)));
    dc_to_bf16_kernel<<<4 * 152, 256, 0, st>>>(h->Dc64, (bf16*)h->Dtc, h->g.nc, h->g.Vc * 9);
    AMG_LAUNCH_CHECK();
    // BF16 planes of the apply's input, sized for the largest supported column count <= max_nrhs
    const int nmax = h->p.max_nrhs >= 16 ? 16 : (h->p.max_nrhs + 3) / 4 * 4;
    h->tc_xbytes = (size_t)h->g.Vc * tc_xpitch(h->g, nmax) * sizeof(bf16);
    AMG_CUDA_TRY(cudaMalloc(&h->tc_x, h->tc_xbytes));
  }
  if (h->p.r_prec == AMG_BF16) {
    const Geom& g = h->g;
    const bool run_ok = g.B[0] % 8 == 0 || 8 % g.B[0] == 0;
    if (g.ntv % 8 || g.Vb % 8 || !run_ok) return AMG_ERR_UNSUPPORTED;
    const size_t n = (size_t)g.Vc * 2 * 2 * g.ntv * g.nagg;
    AMG_CUDA_TRY(cudaMalloc(&h->Rtc, n * sizeof(bf16)));
    r_to_tc_kernel<<<4 * 152, 256, 0, st>>>(h->R64, (bf16*)h->Rtc, g);
    AMG_LAUNCH_CHECK();
  }
  return AMG_OK;
}

void amg_internal_free_tc(amg_coarse* h) {
  cudaFree(h->Dtc);
  cudaFree(h->Rtc);
  cudaFree(h->tc_x);
  h->Dtc = h->Rtc = h->tc_x = nullptr;
}

amg_status amg_internal_export_stored(amg_coarse* h, double2* out) {
  if (!h->Dtc) return AMG_ERR_UNSUPPORTED;
  const size_t n = (size_t)h->g.Vc * 9 * h->g.nc * h->g.nc;
  double2* tmp = nullptr;
  AMG_CUDA_TRY(cudaMalloc(&tmp, n * sizeof(double2)));
  bf16_to_dc_kernel<<<4 * 152, 256, 0, h->last_stream>>>((const bf16*)h->Dtc, tmp, h->g.nc, h->g.Vc * 9);
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
