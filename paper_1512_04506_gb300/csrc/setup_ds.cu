// D_c = R D P assembly (Alg. 5, Eq. cgo via Alg. 7's D P) in pairs of FP32 numbers.
//
// The same rank-6 sums as the FP64 assembly (forward hop x -> x+mu: -1/2 A(x)^dagger Bt(x) with
// A = u^dagger P(x), Bt = u^dagger U_mu(x) P(x+mu); self: P^dagger ((4+m0) + C) P), with every
// number held as an unevaluated sum h + l of two floats (about 47 significant bits) instead of a
// double: on this GPU the FP32 pipes issue about sixty times as many operations per cycle as the
// FP64 pipe, and a product or a sum of such pairs costs a dozen FP32 operations.
//
//   split     a double becomes h + l by integer operations on its IEEE-754 fields: h takes the
//             leading 24 significant bits, l the next 23 (truncation, relative error < 2^-47)
//   product   x y = p + e exactly with p = fl(xh yh), e = fma(xh, yh, -p) (the FMA residual);
//             the first-order terms xh yl + xl yh join e, xl yl (< 2^-46 |x y|) is dropped
//   sum       TwoSum (Knuth): s = fl(a + b) and its exact rounding error, six operations
//
// Accumulation.  The six products of one site (rank 6) are summed into a local pair whose high
// part is exact (TwoSum) and whose low part is a plain FP32 sum of the residuals; the site's pair
// then joins a three-level accumulator (TwoSum on the high and on the low level, the low level's
// errors in a third float), so no rounding error grows with the number of sites.  The result is
// rounded to FP64 once, when it is written.
//
// Work split: one CTA per (block, job) as in the FP64 kernel; sites are visited in an order that
// puts the +mu face last, so one accumulator set serves both the links inside the block (S_mu) and
// those leaving it (F_mu): it is written out and cleared where the face starts.  For the self job
// the tiles that lie wholly in a chirality off-diagonal quadrant are skipped (those entries are not
// used).
#include "amg_internal.cuh"
#include "pipe.cuh"

namespace {

// ------------------------------------------------------------------ pairs of floats
struct pc {  // complex (rh + rl) + i (ih + il)
  float rh, ih, rl, il;
};

// h + l = x to 47 bits, from the fields of x (sign, 11-bit exponent, 52-bit fraction).  |x| below
// 2^-126 gives 0 (and the low part is dropped below 2^-80); |x| must be below 2^127.
__device__ __forceinline__ void split_double(double x, float& h, float& l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const int ef = e - 1023 + 127;  // FP32 biased exponent of the leading bit
  h = ef >= 1 ? __uint_as_float(sgn | ((unsigned)ef << 23) | (unsigned)(m >> 29)) : 0.0f;
  // remaining 29 fraction bits, leading 23 of them: r * 2^(e - 1023 - 46)
  const unsigned r = (unsigned)((m & 0x1FFFFFFFull) >> 6);
  const int es = e - 1023 - 46 + 127;
  const float rf = __fsub_rn(__uint_as_float(0x4B000000u | r), 8388608.0f);  // exact: r < 2^23
  l = es >= 1 ? __fmul_rn(rf, __uint_as_float((unsigned)es << 23)) : 0.0f;      // exact scaling
  if (sgn) l = -l;
}
__device__ __forceinline__ pc split_c(double2 z) {
  pc r;
  split_double(z.x, r.rh, r.rl);
  split_double(z.y, r.ih, r.il);
  return r;
}
__device__ __forceinline__ pc split_conj(double2 z) { return split_c(make_double2(z.x, -z.y)); }

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}
// (sh, sl) += (xh + xl)(yh + yl)
__device__ __forceinline__ void pair_fma(float& sh, float& sl, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  const float e = __fmaf_rn(xh, yh, -p);
  const float c = __fmaf_rn(xh, yl, __fmaf_rn(xl, yh, e));
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, c));
}
// local complex accumulators: acc += a b, acc += conj(a) b
struct lacc {
  float rh, rl, ih, il;
};
__device__ __forceinline__ void lacc_fma(lacc& s, const pc& a, const pc& b) {
  pair_fma(s.rh, s.rl, a.rh, a.rl, b.rh, b.rl);
  pair_fma(s.rh, s.rl, -a.ih, -a.il, b.ih, b.il);
  pair_fma(s.ih, s.il, a.rh, a.rl, b.ih, b.il);
  pair_fma(s.ih, s.il, a.ih, a.il, b.rh, b.rl);
}
__device__ __forceinline__ void lacc_fmac(lacc& s, const pc& a, const pc& b) {
  pair_fma(s.rh, s.rl, a.rh, a.rl, b.rh, b.rl);
  pair_fma(s.rh, s.rl, a.ih, a.il, b.ih, b.il);
  pair_fma(s.ih, s.il, a.rh, a.rl, b.ih, b.il);
  pair_fma(s.ih, s.il, -a.ih, -a.il, b.rh, b.rl);
}
__device__ __forceinline__ pc lacc_value(const lacc& s) {  // normalised pair (|l| <= ulp(h) / 2)
  pc r;
  two_sum(s.rh, s.rl, r.rh, r.rl);
  two_sum(s.ih, s.il, r.ih, r.il);
  return r;
}

// The same operations on (real, imaginary) lane pairs: one packed FP32x2 instruction per pair
// (the FP32 pipes run a packed instruction at the rate of two scalar ones, but it takes one
// issue slot instead of two).
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  const float2 v = __fadd2_rn(s, neg2(a));
  e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(v)))), __fadd2_rn(b, neg2(v)));
}
struct lacc2 {
  float2 h, l;
};
// (sh, sl) += (xh + xl)(yh + yl), lane-wise
__device__ __forceinline__ void pair_fma2(lacc2& s, float2 xh, float2 xl, float2 yh, float2 yl) {
  const float2 p = __fmul2_rn(xh, yh);
  const float2 e = __ffma2_rn(xh, yh, neg2(p));
  const float2 c = __ffma2_rn(xh, yl, __ffma2_rn(xl, yh, e));
  float2 t;
  two_sum2(s.h, p, s.h, t);
  s.l = __fadd2_rn(s.l, __fadd2_rn(t, c));
}
struct gacc2 {
  float2 h, l, ll;
};
__device__ __forceinline__ void gacc2_add(gacc2& g, const lacc2& a) {
  float2 t, u, w, x;
  two_sum2(g.h, a.h, g.h, t);
  two_sum2(g.l, a.l, u, w);
  two_sum2(u, t, g.l, x);
  g.ll = __fadd2_rn(g.ll, __fadd2_rn(w, x));
}

// -b_mu(a, b(a)) z for the one nonzero entry of row a of b_mu (-i sigma_x, -i sigma_y, -i sigma_z, 1):
// b(a) = 1 - a for mu = 0, 1 (off-diagonal), b(a) = a for mu = 2, 3
__device__ __forceinline__ pc neg_b(int mu, int a, const pc& z) {
  pc r;
  if (mu == 0 || (mu == 2 && a == 0)) {  // -(-i) z = i z
    r.rh = -z.ih; r.rl = -z.il; r.ih = z.rh; r.il = z.rl;
  } else if (mu == 2) {                   // -(i) z
    r.rh = z.ih; r.rl = z.il; r.ih = -z.rh; r.il = -z.rl;
  } else if (mu == 1 && a == 1) {         // -(+1) z
    r.rh = -z.rh; r.rl = -z.rl; r.ih = -z.ih; r.il = -z.il;
  } else {                                // mu == 1, a == 0: -(-1) z;  mu == 3: identity
    r = mu == 1 ? z : pc{-z.rh, -z.ih, -z.rl, -z.il};
  }
  return r;
}

// ------------------------------------------------------------------ one (block, job)
struct PairJob {
  long long blk, blk_fwd;
  int job, mu, stride_mu, Bmu, nface;
  pc dd;  // 4 + m0
};
__device__ inline PairJob pair_job(const Geom& g, long long blk, int job, double m0) {
  PairJob J;
  J.blk = blk;
  J.job = job;
  J.mu = job < 4 ? job : 0;
  int Xc[4];
  long long r = blk;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    Xc[m] = (int)(r % g.Lc[m]);
    r /= g.Lc[m];
  }
  J.stride_mu = 1;
  J.Bmu = 1;
#pragma unroll
  for (int m = 0; m < 4; ++m) {  // constant indices only
    if (m < J.mu) J.stride_mu *= g.B[m];
    if (m == J.mu) {
      J.Bmu = g.B[m];
      Xc[m] = (Xc[m] + 1) % g.Lc[m];
    }
  }
  J.blk_fwd = ((long long)(Xc[3] * g.Lc[2] + Xc[2]) * g.Lc[1] + Xc[1]) * g.Lc[0] + Xc[0];
  J.nface = job < 4 ? (int)g.Vb / J.Bmu : 0;  // sites on the +mu face, visited last
  J.dd = pc{0.f, 0.f, 0.f, 0.f};
  split_double(4.0 + m0, J.dd.rh, J.dd.rl);
  return J;
}
// visiting order t -> local site: t = l_mu * nface + r for hop jobs (the face, l_mu = B_mu - 1, last)
__device__ inline int pair_site(const PairJob& J, int t) {
  if (J.job == 4) return t;
  const int lmu = t / J.nface, r = t % J.nface;
  return (r / J.stride_mu) * (J.stride_mu * J.Bmu) + lmu * J.stride_mu + (r % J.stride_mu);
}

// A(x) and Bt(x) of one (site, column) into the chunk's shared arrays; the B columns
// interleaved by tile, column c at (c % TC) * ntc + c / TC, so that the TC columns of consecutive
// tile columns are consecutive float4 words (no shared-memory bank conflicts).
//
// Each value is stored in the two lane-pair forms the contraction multiplies, as two float4 rows
// [k][form][ncp]: A as (a_r, a_r | lo) and (a_i, -a_i | lo), B as (b_r, b_i | lo) and (b_i, b_r | lo),
// so that conj(a) b = (a_r, a_r)(b_r, b_i) + (a_i, -a_i)(b_i, b_r) lane-wise.
template <int TC>
__device__ inline void build_item(const Geom& g, const PairJob& J, const double2* __restrict__ R,
                                  const double2* __restrict__ U, const double2* __restrict__ clov, float4* As,
                                  float4* Bs, int ncp, int ntc, int t, int c, bool valid) {
  float4* Ao = As + c;
  float4* Bo = Bs + (c % TC) * ntc + c / TC;
  auto putA = [&](int k, const pc& v) {
    Ao[(size_t)(2 * k) * ncp] = make_float4(v.rh, v.rh, v.rl, v.rl);
    Ao[(size_t)(2 * k + 1) * ncp] = make_float4(v.ih, -v.ih, v.il, -v.il);
  };
  auto putB = [&](int k, const pc& v) {
    Bo[(size_t)(2 * k) * ncp] = make_float4(v.rh, v.ih, v.rl, v.il);
    Bo[(size_t)(2 * k + 1) * ncp] = make_float4(v.ih, v.rh, v.il, v.rl);
  };
  if (!valid) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      putA(k, pc{0.f, 0.f, 0.f, 0.f});
      putB(k, pc{0.f, 0.f, 0.f, 0.f});
    }
    return;
  }
  const int ntv = g.ntv, mu = J.mu;
  const int sl = pair_site(J, t);
  const long long site = block_site(g, J.blk, sl);
  const int hc = c / ntv, j = c % ntv;
  const double2* Rc = R + ((J.blk * 2 + hc) * (long long)ntv + j) * g.nagg + sl * 6;
  if (J.job == 4) {
    // self: A = P(x), Bt = ((4 + m0) + C(x)) P(x) per chirality
    const double2* C6 = clov + (site * 2 + hc) * 36;
    pc q[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      q[k] = split_conj(Rc[k]);
      putA(k, q[k]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      lacc s{0.f, 0.f, 0.f, 0.f};
      lacc_fma(s, J.dd, q[k]);
#pragma unroll
      for (int kp = 0; kp < 6; ++kp) lacc_fma(s, split_c(C6[k * 6 + kp]), q[kp]);
      putB(k, lacc_value(s));
    }
    return;
  }
  // row a of u^dagger z is z_a for the l columns and -b_mu z_b(a) for the r columns, with
  // b(a) = 1 - a for mu = 0, 1 and b(a) = a for mu = 2, 3; row a is fed by spin b = b(a)
  const int lmu = (sl / J.stride_mu) % J.Bmu;
  const bool face = lmu == J.Bmu - 1;
  const int sn = face ? sl - (J.Bmu - 1) * J.stride_mu : sl + J.stride_mu;
  const long long bn = face ? J.blk_fwd : J.blk;
  const double2* Rn = R + ((bn * 2 + hc) * (long long)ntv + j) * g.nagg + sn * 6;
  const double2* Ul = U + (site * 4 + mu) * 9;
#pragma unroll 1
  for (int b = 0; b < 2; ++b) {
    const int a = (hc == 1 && mu < 2) ? 1 - b : b;
    // A = u^dagger P(x)
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const pc v = split_conj(Rc[b * 3 + col]);
      putA(a * 3 + col, hc == 0 ? v : neg_b(mu, a, v));
    }
    // Bt = u^dagger U_mu(x) P(x + mu)
    pc qn[3];
#pragma unroll
    for (int cp = 0; cp < 3; ++cp) qn[cp] = split_conj(Rn[b * 3 + cp]);
#pragma unroll 1
    for (int col = 0; col < 3; ++col) {
      lacc s{0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int cp = 0; cp < 3; ++cp) lacc_fma(s, split_c(Ul[col * 3 + cp]), qn[cp]);
      const pc z = lacc_value(s);
      putB(a * 3 + col, hc == 0 ? z : neg_b(mu, a, z));
    }
  }
}

// One site's rank-6 product into the tile's accumulators: a local pair sum over the six rows,
// then one three-level addition per entry (lanes: real, imaginary part of the entry).
template <int TA, int TC>
__device__ inline void contract_site(const float4* As, const float4* Bs, int ncp, int ntc, int ta, int tc,
                                     gacc2 (&acc)[TA][TC]) {
  lacc2 loc[TA][TC];
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int jj = 0; jj < TC; ++jj) loc[i][jj] = lacc2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll 1  // rolled: the unrolled rank-6 body overflows the instruction cache
  for (int k = 0; k < 6; ++k) {
    float4 a0[TA], a1[TA], b0[TC], b1[TC];
#pragma unroll
    for (int i = 0; i < TA; ++i) {
      a0[i] = As[(size_t)(2 * k) * ncp + ta * TA + i];
      a1[i] = As[(size_t)(2 * k + 1) * ncp + ta * TA + i];
    }
#pragma unroll
    for (int jj = 0; jj < TC; ++jj) {
      b0[jj] = Bs[(size_t)(2 * k) * ncp + jj * ntc + tc];
      b1[jj] = Bs[(size_t)(2 * k + 1) * ncp + jj * ntc + tc];
    }
#pragma unroll
    for (int i = 0; i < TA; ++i)
#pragma unroll
      for (int jj = 0; jj < TC; ++jj) {
        pair_fma2(loc[i][jj], make_float2(a0[i].x, a0[i].y), make_float2(a0[i].z, a0[i].w),
                  make_float2(b0[jj].x, b0[jj].y), make_float2(b0[jj].z, b0[jj].w));
        pair_fma2(loc[i][jj], make_float2(a1[i].x, a1[i].y), make_float2(a1[i].z, a1[i].w),
                  make_float2(b1[jj].x, b1[jj].y), make_float2(b1[jj].z, b1[jj].w));
      }
  }
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int jj = 0; jj < TC; ++jj) gacc2_add(acc[i][jj], loc[i][jj]);
}

template <int TA, int TC>
__device__ inline void write_tile(double2* P, int nc, int ta, int tc, gacc2 (&acc)[TA][TC]) {
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int jj = 0; jj < TC; ++jj) {
      const int a = ta * TA + i, c = tc * TC + jj;
      const gacc2& v = acc[i][jj];
      if (a < nc && c < nc)
        P[a * nc + c] = make_double2(((double)v.ll.x + (double)v.l.x) + (double)v.h.x,
                                     ((double)v.ll.y + (double)v.l.y) + (double)v.h.y);
      acc[i][jj] = gacc2{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    }
}

// tiles wholly off the chirality diagonal carry nothing the self block uses
template <int TA, int TC>
__device__ inline bool tile_needed(int job, int ntv, int ta, int tc) {
  return !(job == 4 && ((ta * TA + TA <= ntv && tc * TC >= ntv) || (ta * TA >= ntv && tc * TC + TC <= ntv)));
}

// Every thread builds, then every thread contracts (barrier between): the form for nc > 48.
template <int TA, int TC>
__global__ void __launch_bounds__(512)
assemble_pair_kernel(const double2* __restrict__ R, const double2* __restrict__ U,
                     const double2* __restrict__ clov, double2* __restrict__ part, Geom g, double m0,
                     int ncp, int sb_max) {
  extern __shared__ float4 smem4[];
  const int nc = g.nc, Vb = (int)g.Vb;
  float4* As = smem4;  // [sb][6][2 forms][ncp]
  float4* Bs = smem4 + (size_t)sb_max * 12 * ncp;
  const int ntc = ncp / TC, ntiles = ntc * (ncp / TA);
  const int tid = threadIdx.x;
  const int ta = tid / ntc, tc = tid % ntc;
  const PairJob J = pair_job(g, blockIdx.x, blockIdx.y, m0);
  const bool active = tid < ntiles && tile_needed<TA, TC>(J.job, g.ntv, ta, tc);
  gacc2 acc[TA][TC];
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = 0; j < TC; ++j) acc[i][j] = gacc2{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  double2* P0 = part + ((J.blk * 5 + J.job) * 2 + 0) * (long long)nc * nc;
  double2* P1 = P0 + (long long)nc * nc;
  for (int t0 = 0; t0 < Vb; t0 += sb_max) {
    const int nsb = min(sb_max, Vb - t0);
    for (int pr = tid; pr < sb_max * ncp; pr += blockDim.x) {
      const int sb = pr / ncp, c = pr % ncp;
      build_item<TC>(g, J, R, U, clov, As + (size_t)sb * 12 * ncp, Bs + (size_t)sb * 12 * ncp, ncp, ntc, t0 + sb, c,
                     sb < nsb && c < nc);
    }
    __syncthreads();
    for (int sb = 0; sb < nsb; ++sb) {
      if (J.job < 4 && t0 + sb == Vb - J.nface && tid < ntiles) write_tile(P0, nc, ta, tc, acc);  // S_mu
      if (active) contract_site(As + (size_t)sb * 12 * ncp, Bs + (size_t)sb * 12 * ncp, ncp, ntc, ta, tc, acc);
    }
    __syncthreads();
  }
  if (tid < ntiles) write_tile(J.job < 4 ? P1 : P0, nc, ta, tc, acc);  // F_mu, or the self block
}

// Warp-specialised form (nc <= 48): NCW contraction warps (a multiple of four, so that every SM
// sub-partition carries the same share) and four builder warps, with two chunk buffers handed over
// through mbarriers (bounded waits; a wait that runs out sets the timeout bit in *err).
constexpr int kBuilders = 128;
template <int TA, int TC>
__global__ void __launch_bounds__(512)
assemble_pair_ws_kernel(const double2* __restrict__ R, const double2* __restrict__ U,
                        const double2* __restrict__ clov, double2* __restrict__ part, Geom g, double m0, int ncp,
                        int sb, int ncons, unsigned* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  amgpipe::Pipe* pp = reinterpret_cast<amgpipe::Pipe*>(smem_raw);
  float4* buf = reinterpret_cast<float4*>(smem_raw + amgpipe::kPipeBytes);  // [2][A | B][sb][6][2][ncp]
  const size_t half = (size_t)sb * 12 * ncp;
  const int nc = g.nc, Vb = (int)g.Vb;
  const int ntc = ncp / TC, ntiles = ntc * (ncp / TA);
  const int tid = threadIdx.x;
  const PairJob J = pair_job(g, blockIdx.x, blockIdx.y, m0);
  const int nch = (Vb + sb - 1) / sb;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      amgpipe::mbar_init(&pp->full[b], kBuilders);
      amgpipe::mbar_init(&pp->empty[b], ncons);
    }
    pp->abort = 0;
    amgpipe::fence_mbar_init();
  }
  __syncthreads();
  if (tid >= ncons) {
    // builders
    const int bt = tid - ncons;
    for (int ch = 0; ch < nch; ++ch) {
      const int b = ch & 1;
      if (ch >= 2 && !amgpipe::wait_phase(&pp->empty[b], ((ch >> 1) - 1) & 1, pp)) {
        amgpipe::abort_cta(pp, err);
        break;
      }
      const int t0 = ch * sb, nsb = min(sb, Vb - t0);
      float4* Ab = buf + (size_t)b * 2 * half;
      for (int pr = bt; pr < sb * ncp; pr += kBuilders) {
        const int s = pr / ncp, c = pr % ncp;
        build_item<TC>(g, J, R, U, clov, Ab + (size_t)s * 12 * ncp, Ab + half + (size_t)s * 12 * ncp, ncp, ntc,
                       t0 + s, c, s < nsb && c < nc);
      }
      amgpipe::mbar_arrive(&pp->full[b]);
    }
    return;
  }
  // contraction
  const int ta = tid / ntc, tc = tid % ntc;
  const bool tile = tid < ntiles;
  const bool active = tile && tile_needed<TA, TC>(J.job, g.ntv, ta, tc);
  gacc2 acc[TA][TC];
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = 0; j < TC; ++j) acc[i][j] = gacc2{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  double2* P0 = part + ((J.blk * 5 + J.job) * 2 + 0) * (long long)nc * nc;
  double2* P1 = P0 + (long long)nc * nc;
  for (int ch = 0; ch < nch; ++ch) {
    const int b = ch & 1;
    if (!amgpipe::wait_phase(&pp->full[b], (ch >> 1) & 1, pp)) {
      amgpipe::abort_cta(pp, err);
      break;
    }
    const int t0 = ch * sb, nsb = min(sb, Vb - t0);
    const float4* Ab = buf + (size_t)b * 2 * half;
    for (int s = 0; s < nsb; ++s) {
      if (J.job < 4 && t0 + s == Vb - J.nface && tile) write_tile(P0, nc, ta, tc, acc);  // S_mu
      if (active) contract_site(Ab + (size_t)s * 12 * ncp, Ab + half + (size_t)s * 12 * ncp, ncp, ntc, ta, tc, acc);
    }
    amgpipe::mbar_arrive(&pp->empty[b]);
  }
  if (tile) write_tile(J.job < 4 ? P1 : P0, nc, ta, tc, acc);  // F_mu, or the self block
}

// ------------------------------------------------------------------ Gram-Schmidt in pairs
// The FP64 kernel's algorithm (block classical Gram-Schmidt on column blocks of 4, each projection
// applied twice, then the block's columns one by one, again twice) with every value a pair of
// floats.  One CTA of up to 512 threads per aggregate; element n of the aggregate in thread n mod T
// (at most GS_PE elements per thread).  Block sums: pair sums per thread, warp shuffles with pair
// additions (TwoSum on both parts), then one warp over the warps' partial sums.
constexpr int GS_PNB = 4;  // columns per block
constexpr int GS_PKG = 2;  // earlier columns per dot-product round
constexpr int GS_PE = 3;   // elements per thread: aggregates of up to 3 x 512 = 1536 = 6 x 4^4 entries

__device__ __forceinline__ void pair_add(float& h, float& l, float h2, float l2) {
  float s, t, u, w;
  two_sum(h, h2, s, t);
  two_sum(l, l2, u, w);
  t = __fadd_rn(t, u);
  two_sum(s, t, h, l);
  l = __fadd_rn(l, w);
}
__device__ __forceinline__ void pc_add(pc& a, const pc& b) {
  pair_add(a.rh, a.rl, b.rh, b.rl);
  pair_add(a.ih, a.il, b.ih, b.il);
}
__device__ __forceinline__ pc pc_shfl_xor(const pc& a, int o) {
  return pc{__shfl_xor_sync(0xffffffffu, a.rh, o), __shfl_xor_sync(0xffffffffu, a.ih, o),
            __shfl_xor_sync(0xffffffffu, a.rl, o), __shfl_xor_sync(0xffffffffu, a.il, o)};
}
// CTA sum of K complex pairs; every thread gets the sums.  red: [32][K] float4.
template <int K>
__device__ inline void pc_block_sum(pc (&v)[K], float4* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o; o >>= 1) pc_add(v[k], pc_shfl_xor(v[k], o));
  __syncthreads();  // red may still be read by the previous call
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp * K + k] = make_float4(v[k].rh, v[k].ih, v[k].rl, v[k].il);
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      pc t = pc{0.f, 0.f, 0.f, 0.f};
      if (lane < nw) {
        const float4 f = red[lane * K + k];
        t = pc{f.x, f.y, f.z, f.w};
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) pc_add(t, pc_shfl_xor(t, o));
      v[k] = t;
    }
  }
  __syncthreads();
  if (warp == 0)
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (lane == k) red[32 * K + k] = make_float4(v[k].rh, v[k].ih, v[k].rl, v[k].il);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float4 f = red[32 * K + k];
    v[k] = pc{f.x, f.y, f.z, f.w};
  }
}
__device__ __forceinline__ pc pc_mul_sub(const pc& w, const pc& q, const pc& cf) {  // w - q cf
  lacc s{w.rh, w.rl, w.ih, w.il};
  lacc_fma(s, pc{-q.rh, -q.ih, -q.rl, -q.il}, cf);
  return lacc_value(s);
}

__global__ void __launch_bounds__(512) gs_pair_kernel(const double2* __restrict__ tv, double2* __restrict__ R, Geom g,
                                                      unsigned* err) {
  __shared__ float4 red[32 * GS_PKG * GS_PNB + GS_PKG * GS_PNB];
  __shared__ float4 coef[AMG_MAX_NTV * GS_PNB];
  const long long agg = blockIdx.x;
  const long long blk = agg >> 1;
  const int h = (int)(agg & 1);
  const int T = blockDim.x, tid = threadIdx.x, ntv = g.ntv, nagg = g.nagg;
  long long tvoff[GS_PE];
  bool valid[GS_PE];
#pragma unroll
  for (int e = 0; e < GS_PE; ++e) {
    const int n = tid + e * T;
    valid[e] = n < nagg;
    tvoff[e] = 0;
    if (valid[e]) {
      const int sl = n / 6, a = (n % 6) / 3, col = n % 3;
      const long long site = block_site(g, blk, sl);
      tvoff[e] = ((site * 4 + 2 * h + a) * 3 + col) * (long long)ntv;
    }
  }
  double2* Rblk = R + agg * (long long)ntv * nagg;
  const pc zero{0.f, 0.f, 0.f, 0.f};
  pc w[GS_PE][GS_PNB];
  for (int j0 = 0; j0 < ntv; j0 += GS_PNB) {
    const int nb = min(GS_PNB, ntv - j0);
#pragma unroll
    for (int e = 0; e < GS_PE; ++e)
#pragma unroll
      for (int c = 0; c < GS_PNB; ++c) w[e][c] = (valid[e] && c < nb) ? split_c(tv[tvoff[e] + j0 + c]) : zero;
    double n0[GS_PNB];
    {
      pc nn[GS_PNB];
#pragma unroll
      for (int c = 0; c < GS_PNB; ++c) {
        lacc s{0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int e = 0; e < GS_PE; ++e) lacc_fmac(s, w[e][c], w[e][c]);
        nn[c] = lacc_value(s);
      }
      pc_block_sum<GS_PNB>(nn, red);
#pragma unroll
      for (int c = 0; c < GS_PNB; ++c) n0[c] = (double)nn[c].rh + (double)nn[c].rl;
    }
    // projection against the earlier columns (all coefficients from the same vectors), twice
    for (int pass = 0; pass < 2 && j0 > 0; ++pass) {
      for (int k0 = 0; k0 < j0; k0 += GS_PKG) {
        // this thread's (at most GS_PE) products per entry in one unnormalised pair each
        lacc da[GS_PKG * GS_PNB];
#pragma unroll
        for (int q = 0; q < GS_PKG * GS_PNB; ++q) da[q] = lacc{0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int e = 0; e < GS_PE; ++e) {
          if (!valid[e]) continue;
          const int n = tid + e * T;
#pragma unroll
          for (int kk = 0; kk < GS_PKG; ++kk) {
            const pc r = split_c(Rblk[(long long)(k0 + kk) * nagg + n]);  // conj(q_k)
#pragma unroll
            for (int c = 0; c < GS_PNB; ++c) lacc_fma(da[kk * GS_PNB + c], r, w[e][c]);
          }
        }
        pc d[GS_PKG * GS_PNB];
#pragma unroll
        for (int q = 0; q < GS_PKG * GS_PNB; ++q) d[q] = lacc_value(da[q]);
        pc_block_sum<GS_PKG * GS_PNB>(d, red);
#pragma unroll
        for (int q = 0; q < GS_PKG * GS_PNB; ++q)
          if (tid == q && k0 + q / GS_PNB < j0) coef[k0 * GS_PNB + q] = make_float4(d[q].rh, d[q].ih, d[q].rl, d[q].il);
      }
      __syncthreads();
      // w -= sum_k q_k coef_k in unnormalised pairs, renormalised every 8 columns
      lacc wa[GS_PE][GS_PNB];
#pragma unroll
      for (int e = 0; e < GS_PE; ++e)
#pragma unroll
        for (int c = 0; c < GS_PNB; ++c) wa[e][c] = lacc{w[e][c].rh, w[e][c].rl, w[e][c].ih, w[e][c].il};
      for (int k = 0; k < j0; ++k) {
#pragma unroll
        for (int e = 0; e < GS_PE; ++e) {
          if (!valid[e]) continue;
          const int n = tid + e * T;
          const pc q = split_conj(Rblk[(long long)k * nagg + n]);
          const pc mq{-q.rh, -q.ih, -q.rl, -q.il};
#pragma unroll
          for (int c = 0; c < GS_PNB; ++c) {
            const float4 f = coef[k * GS_PNB + c];
            lacc_fma(wa[e][c], mq, pc{f.x, f.y, f.z, f.w});
          }
        }
        if ((k & 7) == 7)
#pragma unroll
          for (int e = 0; e < GS_PE; ++e)
#pragma unroll
            for (int c = 0; c < GS_PNB; ++c) {
              const pc v = lacc_value(wa[e][c]);
              wa[e][c] = lacc{v.rh, v.rl, v.ih, v.il};
            }
      }
#pragma unroll
      for (int e = 0; e < GS_PE; ++e)
#pragma unroll
        for (int c = 0; c < GS_PNB; ++c) w[e][c] = lacc_value(wa[e][c]);
      __syncthreads();
    }
    // orthonormalise inside the block
#pragma unroll
    for (int c = 0; c < GS_PNB; ++c) {
      if (c >= nb) break;
      for (int pass = 0; pass < 2 && c > 0; ++pass) {
        pc d[GS_PNB];
#pragma unroll
        for (int cp = 0; cp < GS_PNB; ++cp) {
          lacc s{0.f, 0.f, 0.f, 0.f};
          if (cp < c)
#pragma unroll
            for (int e = 0; e < GS_PE; ++e) lacc_fmac(s, w[e][cp], w[e][c]);
          d[cp] = lacc_value(s);
        }
        pc_block_sum<GS_PNB>(d, red);
#pragma unroll
        for (int e = 0; e < GS_PE; ++e)
#pragma unroll
          for (int cp = 0; cp < GS_PNB; ++cp)
            if (cp < c) w[e][c] = pc_mul_sub(w[e][c], w[e][cp], d[cp]);
      }
      pc nn[1];
      {
        lacc s{0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int e = 0; e < GS_PE; ++e) lacc_fmac(s, w[e][c], w[e][c]);
        nn[0] = lacc_value(s);
      }
      pc_block_sum<1>(nn, red);
      const double nrm = sqrt((double)nn[0].rh + (double)nn[0].rl);
      if (!(nrm > 1e-12 * sqrt(n0[c]))) {
        if (tid == 0) atomicOr(err, AMG_EBIT_RANK);
      }
      pc inv{0.f, 0.f, 0.f, 0.f};
      split_double(nrm > 0 ? 1.0 / nrm : 0.0, inv.rh, inv.rl);
#pragma unroll
      for (int e = 0; e < GS_PE; ++e) {
        lacc s{0.f, 0.f, 0.f, 0.f};
        lacc_fma(s, inv, w[e][c]);
        w[e][c] = lacc_value(s);
      }
    }
#pragma unroll
    for (int e = 0; e < GS_PE; ++e) {
      if (!valid[e]) continue;
      const int n = tid + e * T;
#pragma unroll
      for (int c = 0; c < GS_PNB; ++c)
        if (c < nb)
          Rblk[(long long)(j0 + c) * nagg + n] =
              make_double2((double)w[e][c].rh + (double)w[e][c].rl, -((double)w[e][c].ih + (double)w[e][c].il));
    }
    __syncthreads();
  }
}

int round_up_i(int a, int b) { return (a + b - 1) / b * b; }
int lcm_i(int a, int b) {
  int x = a, y = b;
  while (y) {
    const int t = x % y;
    x = y;
    y = t;
  }
  return a / x * b;
}

template <int TA, int TC>
amg_status launch_ws(const Geom& g, const double2* R, const double2* U, const double2* clov, double2* part,
                     double m0, unsigned* err, cudaStream_t st) {
  const int ncp = round_up_i(g.nc, lcm_i(TA, TC));
  const int ntiles = (ncp / TA) * (ncp / TC);
  const int ncons = round_up_i(ntiles, 128);
  const int sb = 4;
  const size_t sm = amgpipe::kPipeBytes + (size_t)2 * 2 * sb * 12 * ncp * sizeof(float4);
  AMG_CUDA_TRY(cudaFuncSetAttribute(assemble_pair_ws_kernel<TA, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  assemble_pair_ws_kernel<TA, TC><<<dim3((unsigned)g.Vc, 5), ncons + kBuilders, sm, st>>>(R, U, clov, part, g, m0, ncp,
                                                                                         sb, ncons, err);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

}  // namespace

// Partial sums of the assembly (the layout the combine step reads) in pairs of floats.
amg_status amg_internal_assemble_pair(const Geom& g, const double2* R, const double2* U, const double2* clov,
                                      double2* part, double m0, unsigned* err, cudaStream_t st) {
  if (g.nc <= 48) {
    // tile shape: fewest tile-rows per SM sub-partition (time), at most 384 contraction threads
    struct Shape {
      int ta, tc;
    };
    const Shape shapes[] = {{2, 3}, {1, 5}, {2, 2}, {1, 4}, {1, 2}, {1, 1}};
    int best = -1;
    long long best_cost = 0;
    for (int k = 0; k < 6; ++k) {
      const int ncp = round_up_i(g.nc, lcm_i(shapes[k].ta, shapes[k].tc));
      const int ntiles = (ncp / shapes[k].ta) * (ncp / shapes[k].tc);
      const int warps_per_smsp = (ntiles + 127) / 128;
      if (warps_per_smsp > 3) continue;
      const long long cost = (long long)warps_per_smsp * shapes[k].ta * shapes[k].tc;
      if (best < 0 || cost < best_cost) {
        best = k;
        best_cost = cost;
      }
    }
    switch (best) {
      case 0: return launch_ws<2, 3>(g, R, U, clov, part, m0, err, st);
      case 1: return launch_ws<1, 5>(g, R, U, clov, part, m0, err, st);
      case 2: return launch_ws<2, 2>(g, R, U, clov, part, m0, err, st);
      case 3: return launch_ws<1, 4>(g, R, U, clov, part, m0, err, st);
      case 4: return launch_ws<1, 2>(g, R, U, clov, part, m0, err, st);
      case 5: return launch_ws<1, 1>(g, R, U, clov, part, m0, err, st);
      default: return AMG_ERR_UNSUPPORTED;
    }
  }
  // 2x4 tiles up to nc = 64 (512 threads), every thread builds and contracts
  const int TA = 2, TC = 4;
  const int ncp = round_up_i(g.nc, TC);
  const int ntiles = (ncp / TA) * (ncp / TC);
  const int T = round_up_i(ntiles, 32);
  if (T > 512) return AMG_ERR_UNSUPPORTED;
  int sb = 16;  // sites per chunk: one CTA per SM (the register file), so most of shared memory
  while (sb > 1 && (size_t)sb * 24 * ncp * sizeof(float4) > 200 * 1024) sb >>= 1;
  const size_t sm = (size_t)sb * 24 * ncp * sizeof(float4);
  AMG_CUDA_TRY(cudaFuncSetAttribute(assemble_pair_kernel<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  assemble_pair_kernel<2, 4><<<dim3((unsigned)g.Vc, 5), T, sm, st>>>(R, U, clov, part, g, m0, ncp, sb);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// Gram-Schmidt of every aggregate in pairs of floats; AMG_ERR_UNSUPPORTED when an aggregate has
// more than 1536 entries (the FP64 kernel then serves).
amg_status amg_internal_gs_pair(const Geom& g, const double2* tv, double2* R, unsigned* err, cudaStream_t st) {
  if (g.nagg > GS_PE * 512) return AMG_ERR_UNSUPPORTED;
  int T = round_up_i((g.nagg + GS_PE - 1) / GS_PE, 32);
  if (T < 64) T = 64;
  gs_pair_kernel<<<(unsigned)(g.Vc * 2), T, 0, st>>>(tv, R, g, err);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}
