// Multi-right-hand-side forms of Alg. 2 on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation) for nrhs = 4, 8, 12 or 16 right-hand sides:
//   coarse apply   y_c = D_c x_c   (D_c in BF16 Re/Im planes; Sec. 3 stores D_c in half precision)
//   restriction    y_c = R y       (R in BF16 Re/Im planes, y BF16)
//   prolongation   x   = R^dag x_c (x BF16)
//
// Complex products.  One operand is a pair of real planes (P_re, P_im); the other stays
// complex-interleaved (rows or columns alternate Re, Im of the same right-hand side), so
//   out = P_re . V + P_im . V'
// where V' is V with every (Re, Im) pair replaced by (-Im, Re) (for the product with R^dag, by
// (Im, -Re)).  The pair partner sits in the lane four places away in an mma fragment, so V' costs
// one shuffle and a sign flip per fragment register, and the accumulator holds complete complex
// outputs.
//
// Shared-memory layouts are chosen so that every ldmatrix phase (8 rows of 16 bytes) touches eight
// different 16-byte bank groups:
//   * BF16 rows of D_c and R (stored that way in HBM by the setup): the 16-byte pieces of row r are
//     rotated by rot(r) (tc_rot below);
//   * vectors: rows (apply) or sites (restriction) are placed an odd number of 16-byte units apart.
// All operands arrive by cp.async.bulk into an mbarrier ring filled by one producer warp (pipe.cuh).
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
__device__ inline void ldsm_x4(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ inline void ldsm_x2(unsigned& r0, unsigned& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(smem_addr(p)));
}
__device__ inline void ldsm_x4_trans(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ inline void ldsm_x2_trans(unsigned& r0, unsigned& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(smem_addr(p)));
}

// Rotation of the 16-byte pieces of BF16 row r in a row of P pieces (P = 2, 4, 6 or 8): piece c is
// stored at position (c + tc_rot(r, P)) % P.  For 8 consecutive rows r0 .. r0 + 7 (r0 a multiple of
// 8) and any fixed c, the stored units r P + position are distinct modulo 8.
__host__ __device__ inline int tc_rot(int r, int P) {
  return P == 8 ? (r & 7) : (P == 4 ? ((r >> 1) & 3) : ((r >> 2) & 1));
}
__host__ __device__ inline int tc_pos(int r, int c, int P) { return (c + tc_rot(r, P)) % P; }

// (Re, Im) partner exchange: lane (g, tq) <-> lane (g ^ 1, tq)
__device__ inline unsigned partner(unsigned v) { return __shfl_xor_sync(0xffffffffu, v, 4); }
__device__ inline float partnerf(float v) { return __shfl_xor_sync(0xffffffffu, v, 4); }
constexpr unsigned kNeg2 = 0x80008000u;  // sign bits of two packed BF16

__device__ inline unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  unsigned u;
  memcpy(&u, &v, 4);
  return u;
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

// ------------------------------------------------------------------ coarse apply
// Per coarse site i and stencil block d the stage holds D_c[i][d] (2 planes x nc rows x nc BF16,
// rotated pieces) followed by the BF16 coarse vector of nbr(i, d): nc rows of nrhs (Re, Im) pairs,
// row pitch tc_xunits(nrhs) 16-byte units (odd).  A = D plane (M = nc, K = nc), B = x rows (K = nc,
// N = 2 nrhs interleaved), B' from B by the partner exchange.  Consumer warp w owns output rows
// 16 w .. 16 w + 15 of every site and all right-hand sides.

__host__ __device__ inline int tc_xunits(int nrhs) {
  const int pieces = nrhs / 4;
  return pieces + ((pieces & 1) ? 0 : 1);
}

struct TcApplyArgs {
  const bf16* D;   // [Vc][9][2][nc][nc] BF16 planes, rows with rotated pieces
  const bf16* X;   // [Vc][nc][xunits * 8] BF16 (Re, Im) pairs, see xc_to_bf16_kernel
  const int* nbr;
  float2* y;
  const int* skip;
  unsigned* err;
  Geom g;
  int ns;
};

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
__global__ void __launch_bounds__(160, 1) apply_tc_kernel(const TcApplyArgs a) {
  constexpr int NT = NRHS / 4;  // n-tiles: 8 columns = 4 right-hand sides x (Re, Im)
  constexpr int XU = NRHS / 4 + ((NRHS / 4) & 1 ? 0 : 1);
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int nc = a.g.nc, ns = a.ns, P = nc / 8;
  const unsigned dbytes = (unsigned)(2 * nc * nc * sizeof(bf16));
  const unsigned xbytes = (unsigned)(nc * XU * 16);
  const unsigned chunk = dbytes + xbytes;
  unsigned char* stages = sm + kPipeBytes;
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
      // the neighbour indices of the next site are loaded while the current site's copies are issued
      int nb[9], nx[9];
      if (blockIdx.x < Vc)
        for (int d = 0; d < 9; ++d) nx[d] = __ldg(a.nbr + blockIdx.x * 9LL + d);
      for (long long i = blockIdx.x; i < Vc && !pp->abort; i += gridDim.x) {
#pragma unroll
        for (int d = 0; d < 9; ++d) nb[d] = nx[d];
        if (i + gridDim.x < Vc)
#pragma unroll
          for (int d = 0; d < 9; ++d) nx[d] = __ldg(a.nbr + (i + gridDim.x) * 9 + d);
#pragma unroll
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
          bulk_load(st + dbytes, reinterpret_cast<const unsigned char*>(a.X) + (long long)nb[d] * xbytes, xbytes,
                    &pp->full[s]);
        }
      }
      drain(pp, c, ns);
    }
    return;
  }
  const int w = (threadIdx.x - 32) >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3, q = lane >> 3, li = lane & 7;
  const bool even = !(g & 1);
  // ldmatrix row of this lane: A (non-trans) matrix q = rows 8 (q & 1) .., pieces + (q >> 1);
  // B (trans) matrix q = k rows 8 (q & 1) .., n-tile + (q >> 1)
  const int arow = w * 16 + 8 * (q & 1) + li;
  long long c = 0;
  for (long long i = blockIdx.x; i < Vc; i += gridDim.x) {
    float acc[NT][4], acc2[NT][4];  // products with the Re and the Im plane (two shorter mma chains)
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[t][u] = acc2[t][u] = 0.f;
    for (int d = 0; d < 9; ++d, ++c) {
      const int s = (int)(c % ns);
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], (unsigned)((c / ns) & 1), pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      ok = __all_sync(0xffffffffu, ok);  // the fragment loads and mma below need the whole warp
      if (ok) {
        const unsigned char* Ds = stages + (size_t)s * chunk;
        const unsigned char* Xs = Ds + dbytes;
        for (int ks = 0; ks < nc / 16; ++ks) {
          unsigned are[4], aim[4];
          const unsigned char* ap = Ds + (size_t)arow * nc * 2 + tc_pos(arow, 2 * ks + (q >> 1), P) * 16;
          ldsm_x4(are, ap);
          ldsm_x4(aim, ap + (size_t)nc * nc * 2);
          const unsigned char* bp = Xs + (size_t)(16 * ks + 8 * (q & 1) + li) * XU * 16;
#pragma unroll
          for (int t = 0; t < NT; t += 2) {
            unsigned b[4];
            if (t + 1 < NT) {
              ldsm_x4_trans(b, bp + (t + (q >> 1)) * 16);
            } else {
              ldsm_x2_trans(b[0], b[1], bp + t * 16);
              b[2] = b[3] = 0u;
            }
#pragma unroll
            for (int v = 0; v < 2 && t + v < NT; ++v) {
              const unsigned b0 = b[2 * v], b1 = b[2 * v + 1];
              unsigned p0 = partner(b0), p1 = partner(b1);
              if (even) {
                p0 ^= kNeg2;
                p1 ^= kNeg2;
              }
              mma_bf16(acc[t + v], are, b0, b1);
              mma_bf16(acc2[t + v], aim, p0, p1);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pp->empty[s]);
    }
    // tile t, lane (g, tq): (acc0, acc1) = (Re, Im) of row 16 w + g, right-hand side 4 t + tq;
    // (acc2, acc3) the same for row 16 w + g + 8
    const int row = w * 16 + g;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      a.y[(i * nc + row) * NRHS + 4 * t + tq] = make_float2(acc[t][0] + acc2[t][0], acc[t][1] + acc2[t][1]);
      a.y[(i * nc + row + 8) * NRHS + 4 * t + tq] = make_float2(acc[t][2] + acc2[t][2], acc[t][3] + acc2[t][3]);
    }
  }
}

// ------------------------------------------------------------------ R and P on the tensor cores
// R in BF16 planes, tiled in chunks of 8 block-local sites: Rtc[blk][c][h][p][j][48] with
// p = 0 (Re), 1 (Im).  Within a chunk the 48 aggregate dofs n = 6 sl + d' (site sl = 0..7 of the
// chunk, spin-colour d' = 0..5 of chirality h) are ordered k = 8 d' + sl, so a 16-byte piece of a row
// is one d' over the 8 sites; pieces are rotated by tc_rot(j, 6).
//
// Restriction, per aggregate: Yc^T = Y^T . R^T with A = Y^T (rows: right-hand side x (Re, Im),
// k = 8 d' + sl), B = R plane (k, n = j); A' from A by the partner exchange.  The fine-vector rows
// of the chunk's sites are copied to the stage site by site, 48 nrhs + 16 bytes apart.
// Prolongation, per aggregate: X^T = C^T . conj(R) with A = C^T from x_c (FP32 -> BF16 in
// registers, once per block) and B = R plane (k = j, n = 8 d' + sl).

struct TcRPArgs {
  const bf16* R;       // Rtc
  const void* in;      // restrict: fine BF16 y; prolong: coarse FP32 x_c
  void* out;           // restrict: coarse FP32 y_c; prolong: fine BF16 x
  unsigned* err;
  Geom g;
  int ns;
};

template <int NRHS>
__global__ void __launch_bounds__(160, 1) restrict_tc_kernel(const TcRPArgs a) {
  constexpr int MT = (NRHS + 7) / 8;      // m-tiles per aggregate (16 rows = 8 rhs x (Re, Im))
  constexpr int PIECES = NRHS / 4;        // 16-byte pieces of one fine-vector row
  constexpr int YSITE = 48 * NRHS + 16;   // stage bytes per site (odd number of 16-byte units)
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int ntv = a.g.ntv, ns = a.ns, cpb = (int)(a.g.Vb / 8), NTL = ntv / 8;
  const unsigned rbytes = (unsigned)(2 * 2 * ntv * 48 * sizeof(bf16));
  const unsigned chunk = rbytes + 8 * YSITE;
  unsigned char* stages = sm + kPipeBytes;
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
  const unsigned char* Y = reinterpret_cast<const unsigned char*>(a.in);
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      long long c = 0;
      for (long long blk = blockIdx.x; blk < nblk && !pp->abort; blk += gridDim.x) {
        const long long origin = block_origin(a.g, blk);
        for (int cc = 0; cc < cpb; ++cc, ++c) {
          const int s = (int)(c % ns);
          const long long q = c / ns;
          if (c >= ns && !wait_phase(&pp->empty[s], (unsigned)((q - 1) & 1), pp)) {
            abort_cta(pp, a.err);
            break;
          }
          mbar_expect_tx(&pp->full[s], rbytes + 8 * 48 * NRHS);
          unsigned char* st = stages + (size_t)s * chunk;
          bulk_load(st, a.R + (blk * cpb + cc) * (long long)(rbytes / sizeof(bf16)), rbytes, &pp->full[s]);
          for (int sl = 0; sl < 8; ++sl) {
            const long long site = block_site_fast(a.g, origin, 8 * cc + sl);
            bulk_load(st + rbytes + sl * YSITE, Y + site * 48 * NRHS, 48 * NRHS, &pp->full[s]);
          }
        }
      }
      drain(pp, c, ns);
    }
    return;
  }
  const int w = (threadIdx.x - 32) >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3, q = lane >> 3, li = lane & 7;
  const bool even = !(g & 1);
  const int hw = w / MT, mt = w % MT;  // warp -> (chirality, m-tile)
  const bool half = 2 * mt + 1 >= PIECES;  // m-tile with right-hand sides 8 mt .. 8 mt + 3 only
  // A (trans) matrix q: piece 2 mt + (q & 1) (clamped), d' = 2 ks + (q >> 1), site li
  const int apiece = (2 * mt + (q & 1)) < PIECES ? 2 * mt + (q & 1) : PIECES - 1;
  long long c = 0;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    float acc[4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[t][u] = 0.f;
    for (int cc = 0; cc < cpb; ++cc, ++c) {
      const int s = (int)(c % ns);
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], (unsigned)((c / ns) & 1), pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      ok = __all_sync(0xffffffffu, ok);  // the fragment loads and mma below need the whole warp
      if (ok) {
        const unsigned char* st = stages + (size_t)s * chunk;
        const unsigned char* Ys = st + rbytes;
#pragma unroll
        for (int ks = 0; ks < 3; ++ks) {
          unsigned af[4], ap[4];
          ldsm_x4_trans(af, Ys + li * YSITE + (6 * hw + 2 * ks + (q >> 1)) * (NRHS * 4) + apiece * 16);
          if (half) af[1] = af[3] = 0u;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            ap[u] = partner(af[u]);
            if (even) ap[u] ^= kNeg2;
          }
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            const unsigned char* Rp = st + (size_t)((hw * 2 + p) * ntv) * 96;
#pragma unroll
            for (int t = 0; t < 4; t += 2) {
              if (t >= NTL) break;
              unsigned b[4];
              // B (non-trans) matrix q: rows j = 8 (t + (q >> 1)) + li, k-piece 2 ks + (q & 1)
              if (t + 1 < NTL) {
                const int j = 8 * (t + (q >> 1)) + li;
                ldsm_x4(b, Rp + (size_t)j * 96 + tc_pos(j, 2 * ks + (q & 1), 6) * 16);
              } else {
                const int j = 8 * t + li;
                ldsm_x2(b[0], b[1], Rp + (size_t)j * 96 + tc_pos(j, 2 * ks + (q & 1), 6) * 16);
                b[2] = b[3] = 0u;
              }
#pragma unroll
              for (int v = 0; v < 2; ++v) {
                if (t + v >= NTL) break;
                mma_bf16(acc[t + v], p == 0 ? af : ap, b[2 * v], b[2 * v + 1]);
              }
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pp->empty[s]);
    }
    // tile t, lane (g, tq): rows g (right-hand side 8 mt + g / 2, Re for even g, Im for odd g) and
    // g + 8 (right-hand side + 4); columns j = 8 t + 2 tq, + 1.  Even lanes write column 2 tq, odd
    // lanes column 2 tq + 1, after exchanging one value with the partner.
    float2* yc = reinterpret_cast<float2*>(a.out);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t >= NTL) break;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float x0 = acc[t][2 * u], x1 = acc[t][2 * u + 1];
        const float recv = partnerf(even ? x1 : x0);
        const int r = 8 * mt + (g >> 1) + 4 * u, j = 8 * t + 2 * tq + (g & 1);
        if (r < NRHS)
          yc[((blk * 2 + hw) * ntv + j) * NRHS + r] = even ? make_float2(x0, recv) : make_float2(recv, x1);
      }
    }
  }
}

template <int NRHS>
__global__ void __launch_bounds__(160, 1) prolong_tc_kernel(const TcRPArgs a) {
  constexpr int MT = (NRHS + 7) / 8;
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  const int ntv = a.g.ntv, ns = a.ns, cpb = (int)(a.g.Vb / 8);
  const unsigned chunk = (unsigned)(2 * 2 * ntv * 48 * sizeof(bf16));
  unsigned char* stages = sm + kPipeBytes;
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
  const int w = (threadIdx.x - 32) >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3, q = lane >> 3, li = lane & 7;
  const bool even = !(g & 1);
  const int hw = w / MT, mt = w % MT;
  const int KS = (ntv + 15) / 16;  // k-steps over j (ntv = 8, 16, 24 or 32)
  const float2* xc = reinterpret_cast<const float2*>(a.in);
  __nv_bfloat162* X = reinterpret_cast<__nv_bfloat162*>(a.out);
  long long c = 0;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    // A = C^T and A' (rows: right-hand side 8 mt + g / 2 (+ 4), Re / Im; k = j) from x_c
    unsigned af[2][4], ap[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = 8 * mt + (g >> 1) + 4 * (u & 1), j0 = 16 * ks + 2 * tq + 8 * (u >> 1);
        float lo = 0.f, hi = 0.f, plo = 0.f, phi = 0.f;
        if (ks < KS && r < NRHS) {
          const float2* src = xc + ((blk * 2 + hw) * ntv + j0) * NRHS + r;
          const float2 v0 = j0 < ntv ? src[0] : make_float2(0.f, 0.f);
          const float2 v1 = j0 + 1 < ntv ? src[NRHS] : make_float2(0.f, 0.f);
          lo = even ? v0.x : v0.y;
          hi = even ? v1.x : v1.y;
          plo = even ? v0.y : -v0.x;  // A' rows: (Re -> Im, Im -> -Re) for the product with conj(R)
          phi = even ? v1.y : -v1.x;
        }
        af[ks][u] = pack_bf16(lo, hi);
        ap[ks][u] = pack_bf16(plo, phi);
      }
    const long long origin = block_origin(a.g, blk);
    for (int cc = 0; cc < cpb; ++cc, ++c) {
      const int s = (int)(c % ns);
      bool ok = !pp->abort;
      if (ok && !wait_phase(&pp->full[s], (unsigned)((c / ns) & 1), pp)) {
        abort_cta(pp, a.err);
        ok = false;
      }
      ok = __all_sync(0xffffffffu, ok);  // the fragment loads and mma below need the whole warp
      if (ok) {
        const unsigned char* st = stages + (size_t)s * chunk;
        float acc[6][4];
#pragma unroll
        for (int t = 0; t < 6; ++t)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[t][u] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          if (ks >= KS) break;
          // B (trans) matrix q: rows j = 16 ks + 8 (q & 1) + li (clamped; zeroed past ntv), piece t + (q >> 1)
          int j = 16 * ks + 8 * (q & 1) + li;
          const bool jhi_ok = 16 * ks + 8 < ntv;
          j = j < ntv ? j : ntv - 1;
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            const unsigned char* Rp = st + (size_t)((hw * 2 + p) * ntv + j) * 96;
#pragma unroll
            for (int t = 0; t < 6; t += 2) {
              unsigned b[4];
              ldsm_x4_trans(b, Rp + tc_pos(j, t + (q >> 1), 6) * 16);
              if (!jhi_ok) b[1] = b[3] = 0u;
              mma_bf16(acc[t], p == 0 ? af[ks] : ap[ks], b[0], b[1]);
              mma_bf16(acc[t + 1], p == 0 ? af[ks] : ap[ks], b[2], b[3]);
            }
          }
        }
        // tile t (= d'), lane (g, tq): rows g / g + 8 as in A, columns = sites 2 tq, 2 tq + 1.  After
        // the partner exchange lane (g, tq) holds one BF16 pair w[c] per combination c = 2 (t - t0) + u
        // of a tile pair t0, t0 + 1 and row half u: site 2 tq + (g & 1), right-hand side
        // 8 mt + 4 u + k (k = g / 2).  A 4 x 4 transpose over k (lanes 8 apart) leaves lane k with the
        // four right-hand sides 8 mt + 4 (k & 1) + 0..3 of combination c = k: one 16-byte store.
        const int k = g >> 1, sl = 2 * tq + (g & 1);
        const long long site = block_site_fast(a.g, origin, 8 * cc + sl);
#pragma unroll
        for (int t0 = 0; t0 < 6; t0 += 2) {
          unsigned wv[4];
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            const int t = t0 + (c4 >> 1), u = c4 & 1;
            const float x0 = acc[t][2 * u], x1 = acc[t][2 * u + 1];
            const float recv = partnerf(even ? x1 : x0);
            wv[c4] = even ? pack_bf16(x0, recv) : pack_bf16(recv, x1);
          }
          {
            const bool odd = k & 1;
            const unsigned r0 = __shfl_xor_sync(0xffffffffu, odd ? wv[0] : wv[1], 8);
            const unsigned r1 = __shfl_xor_sync(0xffffffffu, odd ? wv[2] : wv[3], 8);
            if (odd) {
              wv[0] = r0;
              wv[2] = r1;
            } else {
              wv[1] = r0;
              wv[3] = r1;
            }
          }
          {
            const bool hi = k & 2;
            const unsigned r0 = __shfl_xor_sync(0xffffffffu, hi ? wv[0] : wv[2], 16);
            const unsigned r1 = __shfl_xor_sync(0xffffffffu, hi ? wv[1] : wv[3], 16);
            if (hi) {
              wv[0] = r0;
              wv[1] = r1;
            } else {
              wv[2] = r0;
              wv[3] = r1;
            }
          }
          const int r = 8 * mt + 4 * (k & 1), t = t0 + (k >> 1);
          if (r < NRHS)
            *reinterpret_cast<uint4*>(X + (site * 12 + 6 * hw + t) * NRHS + r) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pp->empty[s]);
    }
  }
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

template <int NRHS, bool RESTRICT>
amg_status launch_rp_tc(amg_coarse* h, const void* in, void* out, cudaStream_t st) {
  const Geom& g = h->g;
  const int threads = 32 + 64 * ((NRHS + 7) / 8);
  const size_t rbytes = (size_t)2 * 2 * g.ntv * 48 * sizeof(bf16);
  const size_t chunk = RESTRICT ? rbytes + 8 * (48 * NRHS + 16) : rbytes;
  int ns = (int)((60 * 1024) / chunk);
  ns = ns < 2 ? 2 : (ns > 8 ? 8 : ns);
  const size_t smem = kPipeBytes + ns * chunk;
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  auto kern = RESTRICT ? restrict_tc_kernel<NRHS> : prolong_tc_kernel<NRHS>;
  AMG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  if (per_sm < 1) return AMG_ERR_UNSUPPORTED;
  const long long gmax = (long long)per_sm * sm_count_tc();
  const int grid = (int)(g.Vc < gmax ? g.Vc : gmax);
  TcRPArgs a{(const bf16*)h->Rtc, in, out, h->err, g, ns};
  kern<<<grid, threads, smem, st>>>(a);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
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

size_t tc_xbytes_per_site(const Geom& g, int nrhs) { return (size_t)g.nc * tc_xunits(nrhs) * 16; }

template <int NRHS>
amg_status launch_apply_tc(amg_coarse* h, const void* x, void* y, cudaStream_t st, const int* skip,
                           const double* xscale, void* vout) {
  const int nc = h->g.nc;
  const size_t xsite = tc_xbytes_per_site(h->g, NRHS);
  if ((size_t)h->g.Vc * xsite > h->tc_xbytes) return AMG_ERR_INVALID_ARG;  // nrhs > max_nrhs
  xc_to_bf16_kernel<NRHS><<<4 * 152, 256, 0, st>>>((const float2*)x, (__nv_bfloat162*)h->tc_x, h->g.Vc * nc, xscale,
                                                   (float2*)vout, skip);
  AMG_LAUNCH_CHECK();
  h->launches++;
  const int threads = 32 + 32 * (nc / 16);
  const size_t chunk = (size_t)2 * nc * nc * sizeof(bf16) + xsite;
  // a short ring: more CTAs per SM (each works through its chunks in order) beat deeper prefetch
  int ns = (int)((32 * 1024) / chunk);
  ns = ns < 2 ? 2 : (ns > 6 ? 6 : ns);
  const size_t smem = kPipeBytes + ns * chunk;
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  AMG_CUDA_TRY(cudaFuncSetAttribute(apply_tc_kernel<NRHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_tc_kernel<NRHS>, threads, smem));
  if (per_sm < 1) return AMG_ERR_UNSUPPORTED;
  const long long gmax = (long long)per_sm * sm_count_tc();
  const int grid = (int)(h->g.Vc < gmax ? h->g.Vc : gmax);
  TcApplyArgs a{(const bf16*)h->Dtc, (const bf16*)h->tc_x, h->nbr, (float2*)y, skip, h->err, h->g, ns};
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
    h->tc_xbytes = (size_t)h->g.Vc * tc_xbytes_per_site(h->g, nmax);
    AMG_CUDA_TRY(cudaMalloc(&h->tc_x, h->tc_xbytes));
  }
  if (h->p.r_prec == AMG_BF16) {
    const Geom& g = h->g;
    if (g.ntv % 8 || g.Vb % 8) return AMG_ERR_UNSUPPORTED;
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
