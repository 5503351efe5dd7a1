// Coarse apply y_c = D_c x_c for 4 .. 16 right-hand sides on the 5th-generation tensor cores
// (tcgen05, kind::f16, accumulator in tensor memory), for D_c stored in FP32 or in FP16 with a scale
// per stencil block (Sec. 3's half precision).
//
// Alg. 2 applies D_c inside the coarse solve; with many right-hand sides the product is a dense
// complex contraction per stencil block.  Per coarse site i and block d,
//   [y_re | y_im] += s_D s_x [D_re | D_im]' [[x_re, x_im], [-x_im, x_re]]'_nbr(i,d):
// A = the two planes side by side (M = nc rows of K = 2 nc), B = the neighbour's columns (K x 32:
// columns 0-15 give the real parts of 16 right-hand sides, 16-31 the imaginary parts; fewer
// right-hand sides leave zero columns); ' marks division by a scale: s_D per (site, block), s_x per
// coarse site, so that every scaled entry lies below 2^15 and FP16 holds it.  The FP16 operands are
// split: x' = x_hi + x_lo (both FP16, 22 significant bits together); for FP32 storage also
// D' = D_hi + D_lo with s_D a power of two (exact scaling), split once at setup and kept in HBM as
// FP16 hi and lo planes (the bytes of FP32).  One instruction per K step, tcgen05.mma kind::f16,
// M = 128, N = 64 over [B_hi | B_lo]: FP16 storage gives [A B_hi | A B_lo] in rows 0 .. nc - 1;
// FP32 storage stacks A_hi (rows 0 ..) and A_lo (rows 64 ..) and gives all four products, of which
// A_lo B_lo (below FP32 rounding) is kept as well.
//
// Operands.  The streamed D_c is A and lives in tensor memory (two FP16 per column): with N = 32 an
// A operand in shared memory would be fetched again for every instruction.  A warps (lane
// quadrants 0, 1) copy row q of a bulk-copied block to lane q with tcgen05.st; builder warps write the
// neighbour's columns, split, as the B operand in shared memory
// (K-major, no swizzle: core matrices of 8 rows x 16 bytes, adjacent in K 128 bytes apart, in N
// 16 nc bytes apart).  One thread issues the MMAs; tcgen05.commit tells the builders when an A
// stage and its B buffer may be reused and the epilogue when a block's product is complete.  Each
// block accumulates in its own accumulator (a ring of them), which the epilogue warps scale and
// add up in FP32 registers: the tensor core's FP32 accumulation truncates, and over a whole site's
// instructions that cost about 1e-5 relative.  The A stages let the builders, the accumulator ring
// the MMAs run ahead.
//
// Tensor-memory columns (512 allocated, one CTA per SM): 3 or 4 accumulators of 64 columns, then 4 A
// stages of nc columns (FP32 storage: A_hi in lanes 0 .. nc - 1, A_lo in lanes 64 .., so that one
// M = 128 instruction multiplies both), nc <= 56.
//
// Roles (704 threads): warps 0-15 write the operands in two groups of eight (w / 8) that take
// alternate blocks, so that two blocks are prepared at once; in a group, warps with w % 4 < 2 copy
// the A_hi rows of their lane quadrant and plane, the others (FP32 storage) the A_lo rows; B is
// written by all eight (FP32 storage) or by the four non-A warps (FP16); warps 16-19 (quadrants 0-3) read, scale and sum the block products, the A_lo rows'
// sums handed to the A_hi rows' warps through shared memory once per site, and store y; warp 20
// lane 0 issues the bulk copies; warp 21 allocates tensor memory and lane 0 issues the MMAs.  Every wait is bounded; a wait that runs out raises the CTA's abort flag and sets the
// timeout bit of the error word, after which every role leaves its loop, the MMA thread waits
// (bounded) for its last commit, and tensor memory is freed.
#include "tc_body.cuh"

namespace {
using namespace amgtc;

constexpr int kT5Threads = 704;  // 16 builder warps, 4 epilogue warps, the copy warp, the MMA warp
constexpr int kT5Cols = 512;       // tensor-memory columns allocated

constexpr int kT5MaxStages = 4;  // A stages / B buffers
constexpr int kT5MaxAcc = 8;     // accumulators
struct T5Bars {
  uint64_t aready[kT5MaxStages];  // A stage and B buffer written (the 8 builder warps)
  uint64_t afree[kT5MaxStages];   // the MMAs that read them completed (tcgen05.commit)
  uint64_t accfull[kT5MaxAcc];    // a block's product complete (tcgen05.commit)
  uint64_t accempty[kT5MaxAcc];   // the epilogue has read it (the epilogue warps)
  uint64_t xfull, xempty;         // FP32 storage: the lo rows' site sums handed to the hi rows' warps
  uint64_t done;                  // final commit of the MMA thread
  uint32_t tmem_base;
};
constexpr int kT5BarBytes = 256;
static_assert(sizeof(T5Bars) <= kT5BarBytes, "barrier block");

__device__ inline void tc5_alloc(uint32_t* dst) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
               "r"(kT5Cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tc5_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kT5Cols) : "memory");
}
__device__ inline void tc5_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc5_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ inline void tc5_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
// D[tmem] (+)= A[tmem] B[smem], FP16 operands, FP32 accumulator
__device__ inline void tc5_mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ inline void tc5_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}
__device__ inline void tc5_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ inline void tc5_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major without swizzle: start, leading-dimension byte offset
// (between core matrices adjacent in K), stride-dimension byte offset (adjacent in M / N), and
// the descriptor version bit of this architecture (bit 46).
__device__ inline uint64_t tc5_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((smem_addr(p) & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator, FP16 A and B, both K-major, N, M = 128.
__host__ __device__ constexpr uint32_t tc5_idesc(int n) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ inline bool t5_wait(uint64_t* bar, unsigned parity, Pipe* pp, unsigned* err) {
  if (wait_phase(bar, parity, pp)) return true;
  abort_cta(pp, err);
  return false;
}

// Power of two s with |v| / s < 2^14 for every |v| <= m (1 for m = 0 and for m outside the range
// where s and 1 / s are normal FP32 numbers), from the exponent field of m.
__host__ __device__ inline float pow2_scale(float m) {
  uint32_t b;
  memcpy(&b, &m, 4);
  const int field = (int)((b >> 23) & 0xFF);
  if (field == 0 || field > 200) return 1.0f;
  const int e = field - 126 - 14;  // m < 2^(field - 126)
  if (e < -120 || e > 120) return 1.0f;
  const uint32_t sb = (uint32_t)(e + 127) << 23;
  float s;
  memcpy(&s, &sb, 4);
  return s;
}

__device__ __forceinline__ uint32_t pack_half2(float lo_k, float hi_k) {  // element k in the low half
  const __half2 h = __floats2half2_rn(lo_k, hi_k);
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

// a = hi + lo with hi = FP16(a), lo = FP16(a - hi) for two consecutive K elements (packed)
__device__ __forceinline__ void split_h2(float a0, float a1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a0, a1);
  const float2 hf = __half22float2(h);
  memcpy(&hi, &h, 4);
  lo = pack_half2(a0 - hf.x, a1 - hf.y);
}

struct T5Args {
  const void* D;      // FP16 planes of the scaled entries, [Vc][9][(hi, lo) x (Re, Im) or (Re, Im)][nc][nc]
                      // (16-byte pieces of 8 rotated by tc_rot(r, nc / 8)): FP32 storage split at setup
                      // into hi + lo, FP16 storage as stored
  const float* ds;    // [Vc][9] scale of each stencil block (FP32: power of two; FP16: the stored scale)
  const float* X;     // [Vc][nc][2 nrhs] FP32 coarse rows (already times xscale)
  const float* xs;    // [Vc] power-of-two scale of each site's rows
  const int* nbr;
  float2* y;          // [Vc][nc][nrhs] FP32
  unsigned* err;
  Geom g;
};

// Tensor-memory plan: A stages of nc columns (FP32 storage: A_hi in lanes 0 .. nc - 1 and A_lo in
// lanes 64 .. 64 + nc - 1 of the same columns, so that one M = 128 instruction covers both) and
// 64-column accumulators within 512 columns (accumulators first, A stages from column 64 NACC).
__host__ __device__ constexpr int t5_nst(int nc) { return 4; }  // five (where they fit) measured slower
__host__ __device__ constexpr int t5_nacc(int nc) { return (512 - 4 * nc) / 64 >= 4 ? 4 : 3; }

// Bytes of one B buffer (hi or lo): 32 / 8 column groups x (2 nc / 8) core matrices x 128 bytes.
__host__ __device__ inline unsigned t5_bbytes(int nc) { return 4u * (unsigned)(2 * nc / 8) * 128u; }
__host__ __device__ inline unsigned t5_dbytes(int nc, bool f32) { return (unsigned)((f32 ? 8 : 4) * nc * nc); }
// Coarse rows of the bulk copies: 2 nrhs floats, unpadded (the B writers read them as 8-byte words, 16
// consecutive per half warp, which no pitch makes conflict; padding only added bytes to the copy stream)
__host__ __device__ inline int t5_xpitch(int nrhs) { return 2 * nrhs; }
__host__ __device__ inline unsigned t5_xbytes(int nc, int nrhs) { return (unsigned)(nc * t5_xpitch(nrhs) * 4); }

// The scales of site i's nine blocks, lane d (< 9) holding block d: s_D and s_x of its neighbour.
// Each role loads the next site's while it works on the current one (the loads are dependent:
// neighbour index, then its row scale).
__device__ __forceinline__ void site_scales(const T5Args& a, long long i, int lane, float& sd, float& sx) {
  sd = 1.f;
  sx = 1.f;
  if (lane < 9 && i < a.g.Vc) {
    sd = __ldg(a.ds + i * 9 + lane);
    sx = __ldg(a.xs + __ldg(a.nbr + i * 9 + lane));
  }
}

template <int NC, bool F32>
__global__ void __launch_bounds__(kT5Threads, 1) apply_tc5_kernel(const T5Args a, const int* skip, int ns, int nrhs) {
  if (skip && *skip) return;
  constexpr int K = 2 * NC;
  constexpr int P = NC / 8;                          // 16-byte pieces (8 FP16) per plane row
  constexpr unsigned bbytes = 4u * (unsigned)(K / 8) * 128u;
  constexpr unsigned SBO = (unsigned)(K / 8) * 128u;  // N-adjacent core matrices
  constexpr unsigned dbytes = (unsigned)((F32 ? 8 : 4) * NC * NC);
  constexpr int NST = t5_nst(NC), NACC = t5_nacc(NC);
  static_assert(NST <= kT5MaxStages && NACC <= kT5MaxAcc, "tensor-memory plan");
  constexpr uint32_t AW = (uint32_t)NC;  // tensor-memory columns per A stage
  constexpr uint32_t kAcc = 0, kA = 64u * NACC;
  constexpr int EPI = F32 ? 4 : 2;       // epilogue warps (lane quadrants 0 .. EPI - 1)
  static_assert(kA + NST * AW <= 512, "tensor-memory columns");
  const int XP = t5_xpitch(nrhs);
  const unsigned xbytes = (unsigned)(NC * XP * 4);
  extern __shared__ __align__(128) unsigned char sm[];
  Pipe* pp = reinterpret_cast<Pipe*>(sm);
  T5Bars* tb = reinterpret_cast<T5Bars*>(sm + kPipeBytes);
  unsigned char* bbuf = sm + kPipeBytes + kT5BarBytes;  // B buffers [stage][hi, lo]
  float* xb = reinterpret_cast<float*>(bbuf + 2 * kT5MaxStages * (size_t)bbytes);  // [nc][32] lo-row sums
  unsigned char* stages = bbuf + 2 * kT5MaxStages * (size_t)bbytes + (size_t)NC * 32 * sizeof(float);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ring_init(pp, ns, 8);
  if (threadIdx.x == 0) {
    for (int k = 0; k < NST; ++k) {
      mbar_init(&tb->aready[k], 8);
      mbar_init(&tb->afree[k], 1);
    }
    for (int k = 0; k < NACC; ++k) {
      mbar_init(&tb->accfull[k], 1);
      mbar_init(&tb->accempty[k], EPI);
    }
    mbar_init(&tb->xfull, 2);
    mbar_init(&tb->xempty, 2);
    mbar_init(&tb->done, 1);
    fence_mbar_init();
  }
  if (warp == 21) tc5_alloc(&tb->tmem_base);
  tc5_fence_before();
  __syncthreads();
  tc5_fence_after();
  const uint32_t tmem = tb->tmem_base;
  const Ring rg{pp, stages, ns, dbytes + xbytes};
  const long long i0 = blockIdx.x, step = gridDim.x, Vc = a.g.Vc;

  if (warp == 20) {
    // ---------------------------------------------------------------- bulk copies
    if (lane == 0) {
      RingPos rp;
      // the neighbour indices of the next site load while the current site's copies are issued
      int nb[9], nx[9];
#pragma unroll
      for (int d = 0; d < 9; ++d) nx[d] = __ldg(a.nbr + i0 * 9 + d);
      for (long long i = i0; i < Vc && !pp->abort; i += step) {
#pragma unroll
        for (int d = 0; d < 9; ++d) nb[d] = nx[d];
        if (i + step < Vc)
#pragma unroll
          for (int d = 0; d < 9; ++d) nx[d] = __ldg(a.nbr + (i + step) * 9 + d);
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 9; ++d) {
          unsigned char* st = ring_acquire(rg, rp, dbytes + xbytes, a.err, ok);
          if (!ok) break;
          bulk_load_hint(st, reinterpret_cast<const unsigned char*>(a.D) + (i * 9 + d) * (long long)dbytes, dbytes,
                         &pp->full[rp.s], l2_evict_first_policy());
          bulk_load(st + dbytes, reinterpret_cast<const unsigned char*>(a.X) + (long long)nb[d] * xbytes, xbytes,
                    &pp->full[rp.s]);
          rp.advance(rg.ns);
        }
        if (!ok) break;
      }
      drain(pp, rp.c, ns);
    }
  } else if (warp == 21) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc64 = tc5_idesc(64);
      long long blk = 0;
      bool ok = true;
      for (long long i = i0; i < Vc && ok && !pp->abort; i += step) {
        for (int d = 0; d < 9; ++d, ++blk) {
          const int st = (int)(blk % NST), buf = (int)(blk % NACC);
          // the accumulator of block blk - NACC must have been read, the A stage and B buffer written
          if (blk >= NACC && !t5_wait(&tb->accempty[buf], (unsigned)(((blk / NACC) - 1) & 1), pp, a.err)) {
            ok = false;
            break;
          }
          if (!t5_wait(&tb->aready[st], (unsigned)((blk / NST) & 1), pp, a.err)) {
            ok = false;
            break;
          }
          tc5_fence_after();
          const uint32_t acc = tmem + kAcc + (uint32_t)(buf * 64);
          const uint32_t aa = tmem + kA + (uint32_t)st * AW;
          const unsigned char* bhi = bbuf + (size_t)(2 * st) * bbytes;  // B_lo follows at 4 SBO: N = 64 covers both
#pragma unroll
          for (int ks = 0; ks < K / 16; ++ks) {
            // rows 0 .. nc - 1: [A_hi B_hi | A_hi B_lo]; FP32 rows 64 ..: [A_lo B_hi | A_lo B_lo]
            tc5_mma(acc, aa + 8 * ks, tc5_desc(bhi + ks * 256, 128u, SBO), idesc64, ks > 0 ? 1u : 0u);
          }
          tc5_commit(&tb->afree[st]);
          tc5_commit(&tb->accfull[buf]);
        }
      }
      // every MMA issued has completed before tensor memory is freed
      tc5_commit(&tb->done);
      const long long t0 = clock64();
      while (!mbar_test(&tb->done, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else if (warp >= 16) {
    // ---------------------------------------------------------------- epilogue
    // warp 16 + u reads lane quadrant u: row 32 u + lane for u < 2 (the A_hi rows), row 32 (u - 2) +
    // lane of the A_lo rows for u >= 2 (FP32 storage).  Each block's two 32-column halves times
    // s_D s_x are summed over the site in FP32 registers; at the end of a site the A_lo warps hand
    // their sums to the A_hi warps through shared memory, which add them and store (re, im) pairs.
    const int u = warp - 16;
    if (u < EPI) {
      const bool lo_rows = u >= 2;
      const int q = 32 * (u & 1) + lane;
      const uint32_t lane_off = (uint32_t)(32 * u) << 16;
      long long blk = 0, site = 0;
      bool ok = true;
      float nd, nx;
      site_scales(a, i0, lane, nd, nx);
      for (long long i = i0; i < Vc && ok; i += step, ++site) {
        const float sc_site = nd * nx;
        site_scales(a, i + step, lane, nd, nx);
        float sum[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) sum[c] = 0.f;
        for (int d = 0; d < 9; ++d, ++blk) {
          const int buf = (int)(blk % NACC);
          const float sc = __shfl_sync(0xffffffffu, sc_site, d);
          if (!__all_sync(0xffffffffu, t5_wait(&tb->accfull[buf], (unsigned)((blk / NACC) & 1), pp, a.err))) {
            ok = false;
            break;
          }
          tc5_fence_after();
          uint32_t v[32];
#pragma unroll
          for (int half = 0; half < 2; ++half) {  // columns 0-31 (x B_hi), then 32-63 (x B_lo)
            tc5_ld32(tmem + lane_off + kAcc + (uint32_t)(buf * 64 + 32 * half), v);
            tc5_wait_ld();
#pragma unroll
            for (int c = 0; c < 32; ++c) sum[c] = fmaf(__uint_as_float(v[c]), sc, sum[c]);
          }
          tc5_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tb->accempty[buf]);
        }
        if (!ok) break;
        if (F32) {
          if (lo_rows) {
            if (site > 0 && !__all_sync(0xffffffffu, t5_wait(&tb->xempty, (unsigned)((site - 1) & 1), pp, a.err))) {
              ok = false;
              break;
            }
            if (q < NC)
#pragma unroll
              for (int c = 0; c < 32; ++c) xb[q * 32 + c] = sum[c];
            __syncwarp();
            if (lane == 0) mbar_arrive(&tb->xfull);
            continue;
          }
          if (!__all_sync(0xffffffffu, t5_wait(&tb->xfull, (unsigned)(site & 1), pp, a.err))) {
            ok = false;
            break;
          }
          if (q < NC)
#pragma unroll
            for (int c = 0; c < 32; ++c) sum[c] += xb[q * 32 + c];
          __syncwarp();
          if (lane == 0) mbar_arrive(&tb->xempty);
        }
        if (q < NC) {
          float2* dst = a.y + (i * NC + q) * nrhs;
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c < nrhs) dst[c] = make_float2(sum[c], sum[16 + c]);
        }
      }
    }
  } else {
    // ---------------------------------------------------------------- builders
    // Two groups (w / 8) take alternate blocks.  In a group, A warps (w % 4 < 2): row q = lane of
    // quadrant w % 4, plane (w / 4) % 2; the others (FP32 storage) the A_lo rows of the same plane.
    // B: FP32 storage all eight warps, FP16 storage the four non-A warps.
    const int grp = warp >> 3;
    const bool awarp = (warp & 3) < 2;    // A_hi rows (quadrants 0, 1); the others write B and, for FP32
                                          // storage, the A_lo rows (quadrants 2, 3: lanes 64 + q)
    const bool arow = awarp || F32;
    const int plane = (warp >> 2) & 1;  // 0 = Re, 1 = Im
    const int q = 32 * (warp & 1) + lane;
    const bool row_ok = arow && q < NC;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const int rot = row_ok ? tc_rot(q, P) : 0;
    const size_t lo_off = awarp ? 0 : (size_t)2 * NC * NC * 2;  // the lo planes follow the hi planes
    // B threads: FP32 storage all eight warps of the group (0 .. 255: the A_lo warps would otherwise
    // carry B on top of their rows), FP16 storage the four non-A warps (0 .. 127)
    constexpr int BT = F32 ? 256 : 128;
    const int bt = F32 ? (warp & 7) * 32 + lane : (((warp >> 2) & 1) * 2 + (warp & 3) - 2) * 32 + lane;
    bool ok = true;
    long long blk = 0;
    float nd, nx;
    site_scales(a, i0, lane, nd, nx);
    for (long long i = i0; i < Vc && ok; i += step) {
      const float inv_site = 1.0f / nx;  // a power of two: exact
      site_scales(a, i + step, lane, nd, nx);
      for (int d = 0; d < 9; ++d, ++blk) {
        const float inv_blk = __shfl_sync(0xffffffffu, inv_site, d);
        if ((int)(blk & 1) != grp) continue;
        const int st = (int)(blk % NST);
        RingPos rp;  // ring position of block blk
        rp.c = blk;
        rp.s = (int)(blk % ns);
        rp.ph = (unsigned)((blk / ns) & 1);
        if (!ring_wait(rg, rp, a.err)) {
          ok = false;
          break;
        }
        if (blk >= NST &&
            !__all_sync(0xffffffffu, t5_wait(&tb->afree[st], (unsigned)(((blk / NST) - 1) & 1), pp, a.err))) {
          ok = false;
          break;
        }
        tc5_fence_after();
        const unsigned char* Ds = ring_stage(rg, rp);
        if (arow) {
          // row q of plane `plane` (hi, or lo for the quadrant 2, 3 warps): K columns NC plane ..,
          // two FP16 per column; one 16-byte piece = 8 elements = 4 columns, copied as stored
          const unsigned char* rowp = Ds + lo_off + ((size_t)plane * NC * NC + (size_t)(row_ok ? q : 0) * NC) * 2;
          const uint32_t acol = tmem + lane_off + kA + (uint32_t)st * AW + (uint32_t)(plane * NC / 2);
#pragma unroll
          for (int pc = 0; pc < P; ++pc) {
            int pos = pc + rot;
            pos = pos >= P ? pos - P : pos;
            uint4 f = make_uint4(0u, 0u, 0u, 0u);
            if (row_ok) f = *reinterpret_cast<const uint4*>(rowp + pos * 16);
            asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(acol + (uint32_t)(4 * pc)),
                         "r"(f.x), "r"(f.y), "r"(f.z), "r"(f.w)
                         : "memory");
          }
          tc5_wait_st();
        }
        if (F32 || !awarp) {
          // B (K x 32): column n < 16 = real part of right-hand side n, 16 + n its imaginary part;
          // B = [[x_re, x_im], [-x_im, x_re]]' of the neighbour, split into FP16 hi + lo.  A thread
          // takes rows kk, kk + 1 (kk even) of one right-hand side m: two (re, im) loads, packed
          // splits, four 32-bit positions for hi and for lo
          const float* Xs = reinterpret_cast<const float*>(Ds + dbytes);
          unsigned char* bhi = bbuf + (size_t)(2 * st) * bbytes;
          unsigned char* blo = bhi + bbytes;
          const float inv = inv_blk;
          for (int e = bt; e < NC * 8; e += BT) {
            const int kk = 2 * (e >> 4), m = e & 15;
            float2 x0 = make_float2(0.f, 0.f), x1 = make_float2(0.f, 0.f);
            if (m < nrhs) {
              x0 = *reinterpret_cast<const float2*>(Xs + kk * XP + 2 * m);
              x1 = *reinterpret_cast<const float2*>(Xs + (kk + 1) * XP + 2 * m);
            }
            uint32_t rh, rl, ih, il;
            split_h2(x0.x * inv, x1.x * inv, rh, rl);
            split_h2(x0.y * inv, x1.y * inv, ih, il);
            // (k, n) = (kk, m), (kk, 16 + m), (NC + kk, m), (NC + kk, 16 + m); k and k + 1 share a word
            const unsigned base = (unsigned)(m >> 3) * SBO + (unsigned)(kk >> 3) * 128u + (unsigned)(m & 7) * 16u +
                                  (unsigned)(kk & 7) * 2u;
            const unsigned o1 = base + 2u * SBO, o2 = base + (unsigned)(NC / 8) * 128u, o3 = o2 + 2u * SBO;
            *reinterpret_cast<uint32_t*>(bhi + base) = rh;
            *reinterpret_cast<uint32_t*>(blo + base) = rl;
            *reinterpret_cast<uint32_t*>(bhi + o1) = ih;
            *reinterpret_cast<uint32_t*>(blo + o1) = il;
            *reinterpret_cast<uint32_t*>(bhi + o2) = ih ^ 0x80008000u;
            *reinterpret_cast<uint32_t*>(blo + o2) = il ^ 0x80008000u;
            *reinterpret_cast<uint32_t*>(bhi + o3) = rh;
            *reinterpret_cast<uint32_t*>(blo + o3) = rl;
          }
          fence_async_smem();
        }
        tc5_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tb->aready[st]);
        ring_release(rg, rp);
      }
    }
  }
  tc5_fence_before();
  __syncthreads();
  tc5_fence_after();
  if (warp == 21) tc5_dealloc(tmem);
}

// FP32 coarse vector x (times xscale[r]; the scaled vector also to vout) -> FP32 rows of
// t5_xpitch(nrhs) floats and the power-of-two scale of each site: one warp per site.
__global__ void xc_rows_pow2_kernel(const float2* __restrict__ x, float* __restrict__ X, float* __restrict__ xs,
                                    long long Vc, int nc, int nrhs, const double* __restrict__ xscale,
                                    float2* __restrict__ vout, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int XP = t5_xpitch(nrhs);
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const int per = nc * nrhs;
  for (long long i = w0; i < Vc; i += nw) {
    float m = 0.f;
    for (int e = lane; e < per; e += 32) {
      const int r = e % nrhs;
      float2 v = x[i * per + e];
      if (xscale) {
        const float f = (float)xscale[r];
        v.x *= f;
        v.y *= f;
      }
      if (vout) vout[i * per + e] = v;
      *reinterpret_cast<float2*>(X + (i * nc + e / nrhs) * XP + 2 * r) = v;
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) xs[i] = pow2_scale(m);
  }
}

// Power-of-two scale of every stencil block of the FP32 storage (the FP32 values of the assembled
// FP64 D_c): one warp per block.
__global__ void dc_pow2_scale_kernel(const double2* __restrict__ Dc, float* __restrict__ ds, long long nblk, int nc) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long n = (long long)nc * nc;
  for (long long b = w0; b < nblk; b += nw) {
    float m = 0.f;
    for (long long e = lane; e < n; e += 32) {
      const double2 v = Dc[b * n + e];
      m = fmaxf(m, fmaxf(fabsf((float)v.x), fabsf((float)v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) ds[b] = pow2_scale(m);
  }
}

// FP32 storage for the tcgen05 apply: every entry rounded to FP32, divided by its block's
// power-of-two scale (exact) and split into FP16 hi = FP16(a) and lo = FP16(a - hi); planes
// [Vc][9][hi Re, hi Im, lo Re, lo Im][nc][nc] with rotated 16-byte pieces.
__global__ void dc_f16split_kernel(const double2* __restrict__ Dc, const float* __restrict__ ds, __half* __restrict__ out,
                                   int nc, long long nblk) {
  const long long n2 = (long long)nc * nc, total = nblk * n2;
  const int P = nc / 8;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / n2;
    const int rem = (int)(e % n2), row = rem / nc, col = rem % nc;
    const double2 v = Dc[e];
    const float inv = 1.0f / ds[blk];
    const float re = (float)v.x * inv, im = (float)v.y * inv;
    const __half rh = __float2half_rn(re), ih = __float2half_rn(im);
    const __half rl = __float2half_rn(re - __half2float(rh)), il = __float2half_rn(im - __half2float(ih));
    const int off = row * nc + tc_pos(row, col / 8, P) * 8 + col % 8;
    __half* o = out + blk * 4 * n2 + off;
    o[0] = rh;
    o[n2] = ih;
    o[2 * n2] = rl;
    o[3 * n2] = il;
  }
}

// FP16-scaled D_c (apply layout [Vc][9][nc col][nc row] half2) -> FP16 planes [Vc][9][2][nc][nc]
// with rotated 16-byte pieces (8 elements), the same stored values.
__global__ void dq16_to_planes_kernel(const __half2* __restrict__ Dq, __half* __restrict__ out, int nc, long long nblk) {
  const long long n2 = (long long)nc * nc, total = nblk * n2;
  const int P = nc / 8;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / n2;
    const int rem = (int)(e % n2), row = rem / nc, col = rem % nc;
    const __half2 v = Dq[blk * n2 + (long long)col * nc + row];
    const int off = row * nc + tc_pos(row, col / 8, P) * 8 + col % 8;
    out[blk * 2 * n2 + off] = v.x;
    out[blk * 2 * n2 + n2 + off] = v.y;
  }
}

}  // namespace

// Shared memory of the tcgen05 apply with ns ring stages.
static size_t tc5_smem(int nc, bool f32, int nrhs, int ns) {
  return kPipeBytes + kT5BarBytes + 2 * kT5MaxStages * (size_t)t5_bbytes(nc) + (size_t)nc * 32 * sizeof(float) +
         (size_t)ns * (t5_dbytes(nc, f32) + t5_xbytes(nc, nrhs));
}

bool amg_internal_tc5_supported(const amg_coarse* h) {
  return h->g.nc % 8 == 0 && h->g.nc <= 56 && h->p.vec_prec == AMG_FP32 &&
         (h->p.link_prec == AMG_FP32 || h->p.link_prec == AMG_FP16_SCALED);
}

// Storage for the tcgen05 apply (setup): scales, FP16 planes, coarse rows.
amg_status amg_internal_tc5_prepare(amg_coarse* h, cudaStream_t st) {
  const Geom& g = h->g;
  const int nmax = h->p.max_nrhs < 16 ? h->p.max_nrhs : 16;
  h->tc5_xbytes = 0;
  for (int n = 1; n <= nmax; ++n)  // rows sized for the largest column count
    if ((size_t)g.Vc * t5_xbytes(g.nc, n) > h->tc5_xbytes) h->tc5_xbytes = (size_t)g.Vc * t5_xbytes(g.nc, n);
  AMG_CUDA_TRY(cudaMalloc(&h->tc5_x, h->tc5_xbytes));
  AMG_CUDA_TRY(cudaMalloc(&h->tc5_xs, (size_t)g.Vc * sizeof(float)));
  if (h->p.link_prec == AMG_FP32) {
    AMG_CUDA_TRY(cudaMalloc(&h->tc5_ds, (size_t)g.Vc * 9 * sizeof(float)));
    dc_pow2_scale_kernel<<<4 * amg_sm_count(), 256, 0, st>>>(h->Dc64, h->tc5_ds, g.Vc * 9, g.nc);
    AMG_LAUNCH_CHECK();
    AMG_CUDA_TRY(cudaMalloc(&h->tc5_d16, (size_t)g.Vc * 9 * 4 * g.nc * g.nc * sizeof(__half)));
    dc_f16split_kernel<<<4 * amg_sm_count(), 256, 0, st>>>(h->Dc64, h->tc5_ds, (__half*)h->tc5_d16, g.nc, g.Vc * 9);
    AMG_LAUNCH_CHECK();
  } else {
    AMG_CUDA_TRY(cudaMalloc(&h->tc5_d16, (size_t)g.Vc * 9 * 2 * g.nc * g.nc * sizeof(__half)));
    dq16_to_planes_kernel<<<4 * amg_sm_count(), 256, 0, st>>>((const __half2*)h->Dq, (__half*)h->tc5_d16, g.nc,
                                                                g.Vc * 9);
    AMG_LAUNCH_CHECK();
  }
  return AMG_OK;
}

void amg_internal_free_tc5(amg_coarse* h) {
  cudaFree(h->tc5_x);
  cudaFree(h->tc5_xs);
  cudaFree(h->tc5_ds);
  cudaFree(h->tc5_d16);
  h->tc5_x = nullptr;
  h->tc5_xs = h->tc5_ds = nullptr;
  h->tc5_d16 = nullptr;
  h->tc5_xbytes = 0;
}

template <int NC, bool F32>
static amg_status launch_tc5(amg_coarse* h, const void* x, void* y, int nrhs, cudaStream_t st, const int* skip,
                             const double* xscale, void* vout) {
  if ((size_t)h->g.Vc * t5_xbytes(NC, nrhs) > h->tc5_xbytes) return AMG_ERR_INVALID_ARG;
  xc_rows_pow2_kernel<<<4 * amg_sm_count(), 256, 0, st>>>((const float2*)x, (float*)h->tc5_x, h->tc5_xs, h->g.Vc, NC,
                                                          nrhs, xscale, (float2*)vout, skip);
  AMG_LAUNCH_CHECK();
  h->launches++;
  const size_t stage = t5_dbytes(NC, F32) + t5_xbytes(NC, nrhs);
  // the ring takes what is left of 224 KB: one CTA per SM (it holds all 512 tensor-memory columns)
  int ns = (int)((224 * 1024 - tc5_smem(NC, F32, nrhs, 0)) / stage);
  ns = ns < 2 ? 2 : (ns > kMaxStages ? kMaxStages : ns);
  // an even depth: block b uses stage b % ns, so every stage then belongs to one of the two builder
  // groups (b % 2) and is consumed in order.  With an odd depth a stage alternates between the
  // groups and one group could wait on it for block b + 2 ns while block b + ns of the other is
  // still in flight, and a parity wait cannot tell those phases apart.
  ns &= ~1;
  const size_t smem = tc5_smem(NC, F32, nrhs, ns);
  if (smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  AMG_CUDA_TRY(cudaFuncSetAttribute(apply_tc5_kernel<NC, F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = capped_grid(h, h->g.Vc, amg_sm_count());
  const T5Args a{h->tc5_d16, F32 ? h->tc5_ds : h->Dscale,
                 (const float*)h->tc5_x, h->tc5_xs, h->nbr, (float2*)y, h->err, h->g};
  apply_tc5_kernel<NC, F32><<<grid, kT5Threads, smem, st>>>(a, skip, ns, nrhs);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

template <bool F32>
static amg_status tc5_nc(amg_coarse* h, const void* x, void* y, int nrhs, cudaStream_t st, const int* skip,
                         const double* xscale, void* vout) {
  switch (h->g.nc) {
    case 8: return launch_tc5<8, F32>(h, x, y, nrhs, st, skip, xscale, vout);
    case 16: return launch_tc5<16, F32>(h, x, y, nrhs, st, skip, xscale, vout);
    case 24: return launch_tc5<24, F32>(h, x, y, nrhs, st, skip, xscale, vout);
    case 32: return launch_tc5<32, F32>(h, x, y, nrhs, st, skip, xscale, vout);
    case 40: return launch_tc5<40, F32>(h, x, y, nrhs, st, skip, xscale, vout);
    case 48: return launch_tc5<48, F32>(h, x, y, nrhs, st, skip, xscale, vout);
    case 56: return launch_tc5<56, F32>(h, x, y, nrhs, st, skip, xscale, vout);
    default: return AMG_ERR_UNSUPPORTED;
  }
}

// y = D_c x for FP32 or FP16-scaled storage and 4 <= nrhs <= 16 on tcgen05 (solver extras as in
// amg_internal_apply_ex).
amg_status amg_internal_apply_tc5(amg_coarse* h, const void* x, void* y, int nrhs, cudaStream_t st, const int* skip,
                                  const double* xscale, void* vout) {
  if (!h->tc5_x || nrhs < 1 || nrhs > 16) return AMG_ERR_UNSUPPORTED;
  return h->p.link_prec == AMG_FP32 ? tc5_nc<true>(h, x, y, nrhs, st, skip, xscale, vout)
                                    : tc5_nc<false>(h, x, y, nrhs, st, skip, xscale, vout);
}
