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
// three-level accumulator of one real component
struct gacc {
  float h, l, ll;
};
__device__ __forceinline__ void gacc_add(gacc& g, float h, float l) {
  float s, t, u, w, v, x;
  two_sum(g.h, h, s, t);
  g.h = s;
  two_sum(g.l, l, u, w);
  two_sum(u, t, v, x);
  g.l = v;
  g.ll = __fadd_rn(g.ll, __fadd_rn(w, x));
}
__device__ __forceinline__ double gacc_value(const gacc& g) { return ((double)g.ll + (double)g.l) + (double)g.h; }

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

template <int TA, int TC>
__global__ void __launch_bounds__(512)
assemble_pair_kernel(const double2* __restrict__ R, const double2* __restrict__ U,
                     const double2* __restrict__ clov, double2* __restrict__ part, Geom g, double m0,
                     int ncp, int sb_max) {
  extern __shared__ float4 smem4[];
  const long long blk = blockIdx.x;
  const int job = blockIdx.y;
  const int nc = g.nc, ntv = g.ntv, nagg = g.nagg, Vb = (int)g.Vb;
  float4* As = smem4;  // [sb][6][ncp] (rh, ih, rl, il)
  float4* Bs = smem4 + (size_t)sb_max * 6 * ncp;
  const int ntc = ncp / TC, nta = ncp / TA, ntiles = ntc * nta;
  const int tid = threadIdx.x;
  const int ta = tid / ntc, tc = tid % ntc;
  int Xc[4];
  {
    long long r = blk;
    for (int m = 0; m < 4; ++m) {
      Xc[m] = (int)(r % g.Lc[m]);
      r /= g.Lc[m];
    }
  }
  const int mu = job < 4 ? job : 0;
  int stride_mu = 1, Bmu = 1;
  long long blk_fwd;
  {
    int X[4] = {Xc[0], Xc[1], Xc[2], Xc[3]};
#pragma unroll
    for (int m = 0; m < 4; ++m) {  // constant indices only
      if (m < mu) stride_mu *= g.B[m];
      if (m == mu) {
        Bmu = g.B[m];
        X[m] = (X[m] + 1) % g.Lc[m];
      }
    }
    blk_fwd = ((long long)(X[3] * g.Lc[2] + X[2]) * g.Lc[1] + X[1]) * g.Lc[0] + X[0];
  }
  const int nface = job < 4 ? Vb / Bmu : 0;  // sites on the +mu face, visited last
  // visiting order t -> local site: t = l_mu * nface + r for hop jobs (face: l_mu = B_mu - 1)
  auto site_of = [&](int t) -> int {
    if (job == 4) return t;
    const int lmu = t / nface, r = t % nface;
    return (r / stride_mu) * (stride_mu * Bmu) + lmu * stride_mu + (r % stride_mu);
  };
  // tiles wholly off the chirality diagonal carry nothing the self block uses
  const bool active = tid < ntiles &&
                      !(job == 4 && ((ta * TA + TA <= ntv && tc * TC >= ntv) || (ta * TA >= ntv && tc * TC + TC <= ntv)));
  gacc accr[TA][TC], acci[TA][TC];
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = 0; j < TC; ++j) accr[i][j] = acci[i][j] = gacc{0.f, 0.f, 0.f};
  double2* P0 = part + ((blk * 5 + job) * 2 + 0) * (long long)nc * nc;
  double2* P1 = P0 + (long long)nc * nc;
  auto flush = [&](double2* P) {
    if (tid < ntiles) {
#pragma unroll
      for (int i = 0; i < TA; ++i)
#pragma unroll
        for (int jj = 0; jj < TC; ++jj) {
          const int a = ta * TA + i, c = tc * TC + jj;
          if (a < nc && c < nc) P[a * nc + c] = make_double2(gacc_value(accr[i][jj]), gacc_value(acci[i][jj]));
          accr[i][jj] = acci[i][jj] = gacc{0.f, 0.f, 0.f};
        }
    }
  };
  pc dd{0.f, 0.f, 0.f, 0.f};  // 4 + m0 as a pair
  split_double(4.0 + m0, dd.rh, dd.rl);
  for (int t0 = 0; t0 < Vb; t0 += sb_max) {
    const int nsb = min(sb_max, Vb - t0);
    for (int pr = tid; pr < sb_max * ncp; pr += blockDim.x) {
      const int sb = pr / ncp, c = pr % ncp;
      float4* Ao = As + (size_t)sb * 6 * ncp + c;
      float4* Bo = Bs + (size_t)sb * 6 * ncp + c;
      auto put = [&](float4* o, int k, const pc& v) { o[(size_t)k * ncp] = make_float4(v.rh, v.ih, v.rl, v.il); };
      if (sb >= nsb || c >= nc) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          put(Ao, k, pc{0.f, 0.f, 0.f, 0.f});
          put(Bo, k, pc{0.f, 0.f, 0.f, 0.f});
        }
        continue;
      }
      const int sl = site_of(t0 + sb);
      const long long site = block_site(g, blk, sl);
      const int hc = c / ntv, j = c % ntv;
      const double2* Rc = R + ((blk * 2 + hc) * (long long)ntv + j) * nagg + sl * 6;
      if (job == 4) {
        // self: A = P(x), Bt = ((4 + m0) + C(x)) P(x) per chirality
        const double2* C6 = clov + (site * 2 + hc) * 36;
        pc q[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          q[k] = split_conj(Rc[k]);
          put(Ao, k, q[k]);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          lacc s{0.f, 0.f, 0.f, 0.f};
          lacc_fma(s, dd, q[k]);
#pragma unroll
          for (int kp = 0; kp < 6; ++kp) lacc_fma(s, split_c(C6[k * 6 + kp]), q[kp]);
          put(Bo, k, lacc_value(s));
        }
        continue;
      }
      // row a of u^dagger z is z_a for the l columns and -b_mu z_b(a) for the r columns, with
      // b(a) = 1 - a for mu = 0, 1 and b(a) = a for mu = 2, 3; row a is fed by spin b = b(a)
      const int lmu = (sl / stride_mu) % Bmu;
      const bool face = lmu == Bmu - 1;
      const int sn = face ? sl - (Bmu - 1) * stride_mu : sl + stride_mu;
      const long long bn = face ? blk_fwd : blk;
      const double2* Rn = R + ((bn * 2 + hc) * (long long)ntv + j) * nagg + sn * 6;
      const double2* Ul = U + (site * 4 + mu) * 9;
#pragma unroll 1
      for (int b = 0; b < 2; ++b) {
        const int a = (hc == 1 && mu < 2) ? 1 - b : b;
        // A = u^dagger P(x)
#pragma unroll
        for (int col = 0; col < 3; ++col) {
          const pc v = split_conj(Rc[b * 3 + col]);
          put(Ao, a * 3 + col, hc == 0 ? v : neg_b(mu, a, v));
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
          put(Bo, a * 3 + col, hc == 0 ? z : neg_b(mu, a, z));
        }
      }
    }
    __syncthreads();
    for (int sb = 0; sb < nsb; ++sb) {
      if (job < 4 && t0 + sb == Vb - nface) flush(P0);  // interior links done: S_mu
      if (active) {
        lacc loc[TA][TC];
#pragma unroll
        for (int i = 0; i < TA; ++i)
#pragma unroll
          for (int jj = 0; jj < TC; ++jj) loc[i][jj] = lacc{0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          pc av[TA], bv[TC];
#pragma unroll
          for (int i = 0; i < TA; ++i) {
            const float4 v = As[((size_t)sb * 6 + k) * ncp + ta * TA + i];
            av[i] = pc{v.x, v.y, v.z, v.w};
          }
#pragma unroll
          for (int jj = 0; jj < TC; ++jj) {
            const float4 v = Bs[((size_t)sb * 6 + k) * ncp + tc * TC + jj];
            bv[jj] = pc{v.x, v.y, v.z, v.w};
          }
#pragma unroll
          for (int i = 0; i < TA; ++i)
#pragma unroll
            for (int jj = 0; jj < TC; ++jj) lacc_fmac(loc[i][jj], av[i], bv[jj]);
        }
#pragma unroll
        for (int i = 0; i < TA; ++i)
#pragma unroll
          for (int jj = 0; jj < TC; ++jj) {
            gacc_add(accr[i][jj], loc[i][jj].rh, loc[i][jj].rl);
            gacc_add(acci[i][jj], loc[i][jj].ih, loc[i][jj].il);
          }
      }
    }
    __syncthreads();
  }
  if (job < 4) {
    flush(P1);  // face links: F_mu
  } else {
    flush(P0);  // self; slot 1 is not read for the self job
  }
}

int round_up_i(int a, int b) { return (a + b - 1) / b * b; }

}  // namespace

// Partial sums of the assembly (the layout the combine step reads) in pairs of floats.
amg_status amg_internal_assemble_pair(const Geom& g, const double2* R, const double2* U, const double2* clov,
                                      double2* part, double m0, cudaStream_t st) {
  const bool wide = g.nc > 44;  // 2x2 tiles up to nc = 44 (484 threads), 2x4 tiles up to nc = 64
  const int TA = 2, TC = wide ? 4 : 2;
  const int ncp = round_up_i(g.nc, TC);
  const int ntiles = (ncp / TA) * (ncp / TC);
  const int T = round_up_i(ntiles < 64 ? 64 : ntiles, 32);
  if (T > 512) return AMG_ERR_UNSUPPORTED;
  int sb = 8;
  while (sb > 1 && (size_t)sb * 12 * ncp * sizeof(float4) > 96 * 1024) sb >>= 1;
  const size_t sm = (size_t)sb * 12 * ncp * sizeof(float4);
  dim3 grid((unsigned)g.Vc, 5);
  if (wide) {
    AMG_CUDA_TRY(cudaFuncSetAttribute(assemble_pair_kernel<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    assemble_pair_kernel<2, 4><<<grid, T, sm, st>>>(R, U, clov, part, g, m0, ncp, sb);
  } else {
    AMG_CUDA_TRY(cudaFuncSetAttribute(assemble_pair_kernel<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    assemble_pair_kernel<2, 2><<<grid, T, sm, st>>>(R, U, clov, part, g, m0, ncp, sb);
  }
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}
