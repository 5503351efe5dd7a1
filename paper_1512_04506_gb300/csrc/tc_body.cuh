// Tensor-core bodies of the multi-right-hand-side restriction, coarse apply and prolongation
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation), written over a range of work items and an
// mbarrier ring owned by the caller, so that the standalone kernels (tc.cu) and the fused batch
// (batch.cu) run the same code.
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
//
// Thread roles: a CTA has 32 + 32 ncw threads; lane 0 of warp 0 issues the bulk copies of every
// chunk, warps 1 .. ncw consume (warps a job does not need only wait and release).  The ring
// position runs on across calls, identically in the producer lane and in the consumers.
#pragma once

#include "amg_internal.cuh"
#include "pipe.cuh"

namespace amgtc {
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

// Rotation of the 16-byte pieces of row r in a row of P pieces: piece c is stored at position
// (c + tc_rot(r, P)) % P.  For 8 consecutive rows r0 .. r0 + 7 (r0 a multiple of 8) and any fixed
// c, the stored units r P + position are then distinct modulo 8 (checked for P = 1 .. 16; odd P
// needs no rotation).
__host__ __device__ inline int tc_rot(int r, int P) {
  return P % 8 == 0 ? (r & 7) : P % 4 == 0 ? ((r >> 1) & 3) : P % 2 == 0 ? ((r >> 2) & 1) : 0;
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

// 16-byte units per BF16 coarse row of nrhs (Re, Im) pairs (odd, see above)
__host__ __device__ inline int tc_xunits(int nrhs) {
  const int pieces = nrhs / 4;
  return pieces + ((pieces & 1) ? 0 : 1);
}
// stage bytes of one chunk
__host__ __device__ inline unsigned tc_apply_chunk(int nc, int nrhs) {
  return (unsigned)(2 * nc * nc * 2 + nc * tc_xunits(nrhs) * 16);
}
__host__ __device__ inline unsigned tc_restrict_chunk(int ntv, int nrhs) {
  return (unsigned)(2 * 2 * ntv * 48 * 2 + 8 * (48 * nrhs + 16));
}
__host__ __device__ inline unsigned tc_prolong_chunk(int ntv) { return (unsigned)(2 * 2 * ntv * 48 * 2); }

struct Ring {
  Pipe* pp;
  unsigned char* stages;
  int ns;
  unsigned stride;  // bytes from one stage to the next (at least the chunk of every job using the ring)
};

__device__ inline void ring_init(Pipe* pp, int ns, int consumers) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&pp->full[s], 1);
      mbar_init(&pp->empty[s], consumers);
    }
    pp->abort = 0;
    fence_mbar_init();
  }
}

// Position in the ring: chunk count c, its stage s = c % ns and phase parity ph = (c / ns) & 1,
// advanced without divisions.
struct RingPos {
  long long c = 0;
  int s = 0;
  unsigned ph = 0;
  __device__ void advance(int ns) {
    ++c;
    if (++s == ns) {
      s = 0;
      ph ^= 1u;
    }
  }
};

// Producer side of one chunk: wait until stage s is free, announce the bytes.
__device__ inline unsigned char* ring_acquire(const Ring& rg, const RingPos& rp, unsigned bytes, unsigned* err,
                                              bool& ok) {
  Pipe* pp = rg.pp;
  if (rp.c >= rg.ns && !wait_phase(&pp->empty[rp.s], rp.ph ^ 1u, pp)) {
    abort_cta(pp, err);
    ok = false;
    return nullptr;
  }
  mbar_expect_tx(&pp->full[rp.s], bytes);
  ok = true;
  return rg.stages + (size_t)rp.s * rg.stride;
}
// Consumer side: wait for the chunk at rp (warp-uniform result).
__device__ inline bool ring_wait(const Ring& rg, const RingPos& rp, unsigned* err) {
  Pipe* pp = rg.pp;
  bool ok = !pp->abort;
  if (ok && !wait_phase(&pp->full[rp.s], rp.ph, pp)) {
    abort_cta(pp, err);
    ok = false;
  }
  return __all_sync(0xffffffffu, ok);  // the fragment loads and mma need the whole warp
}
__device__ inline void ring_release(const Ring& rg, const RingPos& rp) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(&rg.pp->empty[rp.s]);
}
__device__ inline const unsigned char* ring_stage(const Ring& rg, const RingPos& rp) {
  return rg.stages + (size_t)rp.s * rg.stride;
}

// ------------------------------------------------------------------ coarse apply
// Per coarse site i and stencil block d the stage holds D_c[i][d] (2 planes x nc rows x nc BF16,
// rotated pieces) followed by the BF16 coarse vector of nbr(i, d): nc rows of nrhs (Re, Im) pairs,
// row pitch tc_xunits(nrhs) 16-byte units (odd).  A = D plane (M = nc, K = nc), B = x rows (K = nc,
// N = 2 nrhs interleaved), B' from B by the partner exchange.  Consumer warp w owns output rows
// 16 w .. 16 w + 15 of every site and all right-hand sides.

struct TcApplyArgs {
  const bf16* D;   // [Vc][9][2][nc][nc] BF16 planes, rows with rotated pieces
  const bf16* X;   // [Vc][nc][xunits * 8] BF16 (Re, Im) pairs
  const int* nbr;
  float2* y;       // [Vc][nc][nrhs] FP32
  unsigned* err;
  Geom g;
};

template <int NRHS>
__device__ void apply_tc_items(const TcApplyArgs& a, const Ring& rg, long long i0, long long i1, long long step,
                               RingPos& rp) {
  constexpr int NT = NRHS / 4;  // n-tiles: 8 columns = 4 right-hand sides x (Re, Im)
  constexpr int XU = NRHS / 4 + ((NRHS / 4) & 1 ? 0 : 1);
  Pipe* pp = rg.pp;
  const int nc = a.g.nc, P = nc / 8;
  const unsigned dbytes = (unsigned)(2 * nc * nc * sizeof(bf16));
  const unsigned xbytes = (unsigned)(nc * XU * 16);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      // the neighbour indices of the next site are loaded while the current site's copies are issued
      int nb[9], nx[9];
      if (i0 < i1)
        for (int d = 0; d < 9; ++d) nx[d] = __ldg(a.nbr + i0 * 9 + d);
      for (long long i = i0; i < i1 && !pp->abort; i += step) {
#pragma unroll
        for (int d = 0; d < 9; ++d) nb[d] = nx[d];
        if (i + step < i1)
#pragma unroll
          for (int d = 0; d < 9; ++d) nx[d] = __ldg(a.nbr + (i + step) * 9 + d);
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 9; ++d) {
          unsigned char* st = ring_acquire(rg, rp, dbytes + xbytes, a.err, ok);
          if (!ok) break;
          bulk_load_hint(st, a.D + (i * 9 + d) * 2LL * nc * nc, dbytes, &pp->full[rp.s], l2_evict_first_policy());
          bulk_load(st + dbytes, reinterpret_cast<const unsigned char*>(a.X) + (long long)nb[d] * xbytes, xbytes,
                    &pp->full[rp.s]);
          rp.advance(rg.ns);
        }
        if (!ok) break;
      }
    }
    return;
  }
  const int w = warp - 1;
  const int KS = (nc + 15) / 16;  // m-tiles and k-steps (nc a multiple of 8: the last may be half)
  const bool active = w < KS;
  const int g = lane >> 2, tq = lane & 3, q = lane >> 3, li = lane & 7;
  const bool even = !(g & 1);
  // ldmatrix row of this lane: A (non-trans) matrix q = rows 8 (q & 1) .., pieces + (q >> 1);
  // B (trans) matrix q = k rows 8 (q & 1) .., n-tile + (q >> 1).  Rows past nc are clamped (their
  // results are not stored); k columns past nc are zeroed in A.
  const int arow = min(w * 16 + 8 * (q & 1) + li, nc - 1);
  for (long long i = i0; i < i1; i += step) {
    float acc[NT][4], acc2[NT][4];  // products with the Re and the Im plane (two shorter mma chains)
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[t][u] = acc2[t][u] = 0.f;
    for (int d = 0; d < 9; ++d) {
      const bool ok = ring_wait(rg, rp, a.err);
      if (ok && active) {
        const unsigned char* Ds = ring_stage(rg, rp);
        const unsigned char* Xs = Ds + dbytes;
        for (int ks = 0; ks < KS; ++ks) {
          unsigned are[4], aim[4];
          const int apc = min(2 * ks + (q >> 1), P - 1);
          const unsigned char* ap = Ds + (size_t)arow * nc * 2 + tc_pos(arow, apc, P) * 16;
          ldsm_x4(are, ap);
          ldsm_x4(aim, ap + (size_t)nc * nc * 2);
          if (16 * ks + 8 >= nc) are[2] = are[3] = aim[2] = aim[3] = 0u;
          const unsigned char* bp = Xs + (size_t)min(16 * ks + 8 * (q & 1) + li, nc - 1) * XU * 16;
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
      ring_release(rg, rp);
      rp.advance(rg.ns);
    }
    // tile t, lane (g, tq): (acc0, acc1) = (Re, Im) of row 16 w + g, right-hand side 4 t + tq;
    // (acc2, acc3) the same for row 16 w + g + 8
    if (active) {
      const int row = w * 16 + g;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        a.y[(i * nc + row) * NRHS + 4 * t + tq] = make_float2(acc[t][0] + acc2[t][0], acc[t][1] + acc2[t][1]);
        if (row + 8 < nc)
          a.y[(i * nc + row + 8) * NRHS + 4 * t + tq] =
              make_float2(acc[t][2] + acc2[t][2], acc[t][3] + acc2[t][3]);
      }
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
  const bf16* R;          // Rtc
  const void* in;         // restrict: fine BF16 y; prolong: coarse FP32 x_c
  void* out;              // restrict: coarse FP32 y_c; prolong: fine BF16 x
  __nv_bfloat162* rows;   // restrict only, optional: y_c also / instead as BF16 rows (apply input)
  bool fp32_out;          // restrict: write the FP32 y_c to out
  unsigned* err;
  Geom g;
};

template <int NRHS>
__device__ void restrict_tc_items(const TcRPArgs& a, const Ring& rg, long long i0, long long i1, long long step,
                                  RingPos& rp) {
  constexpr int MT = (NRHS + 7) / 8;      // m-tiles per aggregate (16 rows = 8 rhs x (Re, Im))
  constexpr int PIECES = NRHS / 4;        // 16-byte pieces of one fine-vector row
  constexpr int YSITE = 48 * NRHS + 16;   // stage bytes per site (odd number of 16-byte units)
  constexpr int XPITCH = 4 * (NRHS / 4 + ((NRHS / 4) & 1 ? 0 : 1));  // pairs per BF16 coarse row
  Pipe* pp = rg.pp;
  const int ntv = a.g.ntv, cpb = (int)(a.g.Vb / 8), NTL = (ntv + 7) / 8;  // ntv a multiple of 4
  const unsigned rbytes = (unsigned)(2 * 2 * ntv * 48 * sizeof(bf16));
  const unsigned char* Y = reinterpret_cast<const unsigned char*>(a.in);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      for (long long blk = i0; blk < i1 && !pp->abort; blk += step) {
        const long long origin = block_origin(a.g, blk);
        bool ok = true;
        for (int cc = 0; cc < cpb; ++cc) {
          unsigned char* st = ring_acquire(rg, rp, rbytes + 8 * 48 * NRHS, a.err, ok);
          if (!ok) break;
          bulk_load_hint(st, a.R + (blk * cpb + cc) * (long long)(rbytes / sizeof(bf16)), rbytes, &pp->full[rp.s],
                         l2_evict_first_policy());
          for (int sl = 0; sl < 8; ++sl) {
            const long long site = block_site_fast(a.g, origin, 8 * cc + sl);
            bulk_load(st + rbytes + sl * YSITE, Y + site * 48 * NRHS, 48 * NRHS, &pp->full[rp.s]);
          }
          rp.advance(rg.ns);
        }
        if (!ok) break;
      }
    }
    return;
  }
  const int w = warp - 1;
  const bool active = w < 2 * MT;
  const int g = lane >> 2, tq = lane & 3, q = lane >> 3, li = lane & 7;
  const bool even = !(g & 1);
  const int hw = w / MT, mt = w % MT;  // warp -> (chirality, m-tile)
  const bool half = 2 * mt + 1 >= PIECES;  // m-tile with right-hand sides 8 mt .. 8 mt + 3 only
  // A (trans) matrix q: piece 2 mt + (q & 1) (clamped), d' = 2 ks + (q >> 1), site li
  const int apiece = (2 * mt + (q & 1)) < PIECES ? 2 * mt + (q & 1) : PIECES - 1;
  for (long long blk = i0; blk < i1; blk += step) {
    float acc[4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[t][u] = 0.f;
    for (int cc = 0; cc < cpb; ++cc) {
      const bool ok = ring_wait(rg, rp, a.err);
      if (ok && active) {
        const unsigned char* st = ring_stage(rg, rp);
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
              // B (non-trans) matrix q: rows j = 8 (t + (q >> 1)) + li, k-piece 2 ks + (q & 1); rows past
              // ntv (last tile when ntv % 8 = 4) read finite data of the stage and are not stored
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
      ring_release(rg, rp);
      rp.advance(rg.ns);
    }
    // tile t, lane (g, tq): rows g (right-hand side 8 mt + g / 2, Re for even g, Im for odd g) and
    // g + 8 (right-hand side + 4); columns j = 8 t + 2 tq, + 1.  Even lanes write column 2 tq, odd
    // lanes column 2 tq + 1, after exchanging one value with the partner.
    if (active) {
      float2* yc = reinterpret_cast<float2*>(a.out);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (t >= NTL) break;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const float x0 = acc[t][2 * u], x1 = acc[t][2 * u + 1];
          const float recv = partnerf(even ? x1 : x0);
          const int r = 8 * mt + (g >> 1) + 4 * u, j = 8 * t + 2 * tq + (g & 1);
          if (r < NRHS && j < ntv) {
            const float2 v = even ? make_float2(x0, recv) : make_float2(recv, x1);
            if (a.fp32_out) yc[((blk * 2 + hw) * ntv + j) * NRHS + r] = v;
            if (a.rows) a.rows[((blk * 2 + hw) * ntv + j) * XPITCH + r] = __floats2bfloat162_rn(v.x, v.y);
          }
        }
      }
    }
  }
}

template <int NRHS>
__device__ void prolong_tc_items(const TcRPArgs& a, const Ring& rg, long long i0, long long i1, long long step,
                                 RingPos& rp) {
  constexpr int MT = (NRHS + 7) / 8;
  Pipe* pp = rg.pp;
  const int ntv = a.g.ntv, cpb = (int)(a.g.Vb / 8);
  const unsigned chunk = (unsigned)(2 * 2 * ntv * 48 * sizeof(bf16));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      for (long long blk = i0; blk < i1 && !pp->abort; blk += step) {
        bool ok = true;
        for (int cc = 0; cc < cpb; ++cc) {
          unsigned char* st = ring_acquire(rg, rp, chunk, a.err, ok);
          if (!ok) break;
          bulk_load_hint(st, a.R + (blk * cpb + cc) * (long long)(chunk / sizeof(bf16)), chunk, &pp->full[rp.s],
                         l2_evict_first_policy());
          rp.advance(rg.ns);
        }
        if (!ok) break;
      }
    }
    return;
  }
  const int w = warp - 1;
  const bool active = w < 2 * MT;
  const int g = lane >> 2, tq = lane & 3, q = lane >> 3, li = lane & 7;
  const bool even = !(g & 1);
  const int hw = w / MT, mt = w % MT;
  const int KS = (ntv + 15) / 16;  // k-steps over j (ntv a multiple of 4, at most 32); A is zero past ntv
  const float2* xc = reinterpret_cast<const float2*>(a.in);
  __nv_bfloat162* X = reinterpret_cast<__nv_bfloat162*>(a.out);
  for (long long blk = i0; blk < i1; blk += step) {
    // A = C^T and A' (rows: right-hand side 8 mt + g / 2 (+ 4), Re / Im; k = j) from x_c
    unsigned af[2][4], ap[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = 8 * mt + (g >> 1) + 4 * (u & 1), j0 = 16 * ks + 2 * tq + 8 * (u >> 1);
        float lo = 0.f, hi = 0.f, plo = 0.f, phi = 0.f;
        if (active && ks < KS && r < NRHS) {
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
    for (int cc = 0; cc < cpb; ++cc) {
      const bool ok = ring_wait(rg, rp, a.err);
      if (ok && active) {
        const unsigned char* st = ring_stage(rg, rp);
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
      ring_release(rg, rp);
      rp.advance(rg.ns);
    }
  }
}


// ------------------------------------------------------------------ FP32 coarse apply, 3 x TF32
// y_c = D_c x_c for FP32 D_c and nrhs = 4 .. 16 right-hand sides on the tensor cores with FP32
// accuracy: every FP32 operand v is split into v_hi = tf32(v) and v_lo = tf32(v - v_hi) and the
// product is accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo term and the
// rounding of v_lo are below FP32's own rounding).  mma.sync m16n8k8 (TF32 in, FP32 accumulate).
// The stage holds D_c[i][d] as two FP32 planes of nc rows (16-byte pieces rotated by tc_rot(r, nc/4))
// and the neighbour's FP32 coarse rows, tf32_xpitch(nrhs) floats apart (a pitch that is 8 or 24
// modulo 32 words, so the B-fragment loads hit distinct banks).  Complex products as in the BF16
// apply (the partner exchange).

__host__ __device__ inline int tf32_xpitch(int nrhs) { return 2 * nrhs + (nrhs % 8 == 0 ? 8 : 0); }
__host__ __device__ inline unsigned tf32_apply_chunk(int nc, int nrhs) {
  return (unsigned)(8 * nc * nc + nc * tf32_xpitch(nrhs) * 4);
}

__device__ inline unsigned tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ inline void split_tf32(unsigned bits, unsigned& hi, unsigned& lo) {
  const float x = __uint_as_float(bits);
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}
__device__ inline void mma_tf32(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct TfApplyArgs {
  const float* D;  // [Vc][9][2][nc][nc] FP32 planes, rows with rotated pieces
  const float* X;  // [Vc][nc][tf32_xpitch(nrhs)] FP32 coarse rows
  const int* nbr;
  float2* y;       // [Vc][nc][nrhs] FP32
  unsigned* err;
  Geom g;
};

template <int NRHS>
__device__ void apply_tf32_items(const TfApplyArgs& a, const Ring& rg, long long i0, long long i1, long long step,
                                 RingPos& rp) {
  constexpr int NT = NRHS / 4;  // n-tiles of 8 columns = 4 right-hand sides x (Re, Im)
  constexpr int XP = 2 * NRHS + (NRHS % 8 == 0 ? 8 : 0);
  Pipe* pp = rg.pp;
  const int nc = a.g.nc, P = nc / 4;
  const unsigned dbytes = (unsigned)(8 * nc * nc);
  const unsigned xbytes = (unsigned)(nc * XP * 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      int nb[9], nx[9];
      if (i0 < i1)
        for (int d = 0; d < 9; ++d) nx[d] = __ldg(a.nbr + i0 * 9 + d);
      for (long long i = i0; i < i1 && !pp->abort; i += step) {
#pragma unroll
        for (int d = 0; d < 9; ++d) nb[d] = nx[d];
        if (i + step < i1)
#pragma unroll
          for (int d = 0; d < 9; ++d) nx[d] = __ldg(a.nbr + (i + step) * 9 + d);
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 9; ++d) {
          unsigned char* st = ring_acquire(rg, rp, dbytes + xbytes, a.err, ok);
          if (!ok) break;
          bulk_load_hint(st, a.D + (i * 9 + d) * 2LL * nc * nc, dbytes, &pp->full[rp.s], l2_evict_first_policy());
          bulk_load(st + dbytes, reinterpret_cast<const unsigned char*>(a.X) + (long long)nb[d] * xbytes, xbytes,
                    &pp->full[rp.s]);
          rp.advance(rg.ns);
        }
        if (!ok) break;
      }
    }
    return;
  }
  const int w = warp - 1;
  const int MTN = (nc + 15) / 16;  // m-tiles (the last may be half); k-steps of 8: nc / 8
  const bool active = w < MTN;
  const int g = lane >> 2, tq = lane & 3, q = lane >> 3, li = lane & 7;
  const unsigned neg = (g & 1) ? 0u : 0x80000000u;  // partner exchange: even columns take -Im
  const int arow = min(w * 16 + 8 * (q & 1) + li, nc - 1);
  for (long long i = i0; i < i1; i += step) {
    float acc[NT][4], acc2[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[t][u] = acc2[t][u] = 0.f;
    for (int d = 0; d < 9; ++d) {
      const bool ok = ring_wait(rg, rp, a.err);
      if (ok && active) {
        const unsigned char* Ds = ring_stage(rg, rp);
        const float* Xs = reinterpret_cast<const float*>(Ds + dbytes);
        for (int ks = 0; ks < nc / 8; ++ks) {
          unsigned are[4], aim[4], arh[4], arl[4], aih[4], ail[4];
          const unsigned char* ap = Ds + (size_t)arow * nc * 4 + tc_pos(arow, 2 * ks + (q >> 1), P) * 16;
          ldsm_x4(are, ap);
          ldsm_x4(aim, ap + (size_t)nc * nc * 4);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            split_tf32(are[u], arh[u], arl[u]);
            split_tf32(aim[u], aih[u], ail[u]);
          }
          const float* x0 = Xs + (size_t)(8 * ks + tq) * XP + g;
          const float* x1 = x0 + 4 * XP;
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const unsigned b0 = __float_as_uint(x0[8 * t]), b1 = __float_as_uint(x1[8 * t]);
            const unsigned p0 = partner(b0) ^ neg, p1 = partner(b1) ^ neg;
            unsigned bh0, bl0, bh1, bl1, ph0, pl0, ph1, pl1;
            split_tf32(b0, bh0, bl0);
            split_tf32(b1, bh1, bl1);
            split_tf32(p0, ph0, pl0);
            split_tf32(p1, ph1, pl1);
            mma_tf32(acc[t], arh, bh0, bh1);
            mma_tf32(acc[t], arh, bl0, bl1);
            mma_tf32(acc[t], arl, bh0, bh1);
            mma_tf32(acc2[t], aih, ph0, ph1);
            mma_tf32(acc2[t], aih, pl0, pl1);
            mma_tf32(acc2[t], ail, ph0, ph1);
          }
        }
      }
      ring_release(rg, rp);
      rp.advance(rg.ns);
    }
    if (active) {
      const int row = w * 16 + g;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (row < nc)
          a.y[(i * nc + row) * NRHS + 4 * t + tq] = make_float2(acc[t][0] + acc2[t][0], acc[t][1] + acc2[t][1]);
        if (row + 8 < nc)
          a.y[(i * nc + row + 8) * NRHS + 4 * t + tq] =
              make_float2(acc[t][2] + acc2[t][2], acc[t][3] + acc2[t][3]);
      }
    }
  }
}

}  // namespace amgtc
