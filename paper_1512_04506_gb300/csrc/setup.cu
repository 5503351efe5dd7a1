// Setup of the restriction and the coarse-grid operator (Alg. 5), in FP64.
//
//   clover_kernel    C(x) = c_sw (i/4) sum sigma_{mu nu} F_{mu nu}(x), per chirality (Alg. 7's C^{hh})
//   gs_kernel        block classical Gram-Schmidt per aggregate (Sec. 3, "Gram-Schmidt on aggregates")
//   assemble_kernel  self and forward blocks of D_c = R D P (Eq. cgo via Alg. 7's D P), as sums
//                    over links of small rank-6 products
//   combine_kernel   D_c blocks from the partial sums; backward blocks by Eq. dagger
//   quantize_*       D_c and R to the storage precisions of the applies (Sec. 3: half precision D_c)
#include "amg_internal.cuh"

#include <stdio.h>
#include <stdlib.h>
#include <vector>

namespace {

// ------------------------------------------------------------------ SU(3) helpers
struct M3 {
  double2 e[9];
};

__device__ inline M3 load_link(const double2* __restrict__ U, long long s, int mu) {
  M3 m;
  const double2* p = U + (s * 4 + mu) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k] = p[k];
  return m;
}
__device__ inline M3 mm(const M3& a, const M3& b) {  // a b
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma(s, a.e[i * 3 + k], b.e[k * 3 + j]);
      c.e[i * 3 + j] = s;
    }
  return c;
}
__device__ inline M3 mmd(const M3& a, const M3& b) {  // a b^dagger
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma(s, a.e[i * 3 + k], cconj(b.e[j * 3 + k]));
      c.e[i * 3 + j] = s;
    }
  return c;
}
__device__ inline M3 mdm(const M3& a, const M3& b) {  // a^dagger b
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cfmac(s, a.e[k * 3 + i], b.e[k * 3 + j]);
      c.e[i * 3 + j] = s;
    }
  return c;
}

__device__ inline long long shifted(const Geom& g, const int* c, int mu, int dmu, int nu, int dnu) {
  int x[4] = {c[0], c[1], c[2], c[3]};
  x[mu] = (x[mu] + dmu + g.L[mu]) % g.L[mu];
  if (dnu) x[nu] = (x[nu] + dnu + g.L[nu]) % g.L[nu];
  return site_index(g.L, x[0], x[1], x[2], x[3]);
}

// F_{mu nu}(x) = (Q - Q^dagger)/8 with Q the four counter-clockwise leaves at x.
__device__ M3 field_strength(const double2* __restrict__ U, const Geom& g, const int* c, long long s,
                             int mu, int nu) {
  const long long xpm = shifted(g, c, mu, 1, nu, 0), xpn = shifted(g, c, nu, 1, mu, 0);
  const long long xmm = shifted(g, c, mu, -1, nu, 0), xmn = shifted(g, c, nu, -1, mu, 0);
  const long long xpn_mm = shifted(g, c, mu, -1, nu, 1), xmm_mn = shifted(g, c, mu, -1, nu, -1);
  const long long xmn_pm = shifted(g, c, mu, 1, nu, -1);
  const M3 Umx = load_link(U, s, mu), Unx = load_link(U, s, nu);
  // leaf 1: U_mu(x) U_nu(x+mu) [U_nu(x) U_mu(x+nu)]^dagger
  M3 Q = mmd(mm(Umx, load_link(U, xpm, nu)), mm(Unx, load_link(U, xpn, mu)));
  // leaf 2: U_nu(x) [U_nu(x-mu) U_mu(x+nu-mu)]^dagger U_mu(x-mu)
  const M3 Umxmm = load_link(U, xmm, mu);
  M3 t = mm(mmd(Unx, mm(load_link(U, xmm, nu), load_link(U, xpn_mm, mu))), Umxmm);
#pragma unroll
  for (int k = 0; k < 9; ++k) Q.e[k] = cadd(Q.e[k], t.e[k]);
  // leaf 3: [U_nu(x-mu-nu) U_mu(x-mu)]^dagger [U_mu(x-mu-nu) U_nu(x-nu)]
  const M3 Unxmn = load_link(U, xmn, nu);
  t = mdm(mm(load_link(U, xmm_mn, nu), Umxmm), mm(load_link(U, xmm_mn, mu), Unxmn));
#pragma unroll
  for (int k = 0; k < 9; ++k) Q.e[k] = cadd(Q.e[k], t.e[k]);
  // leaf 4: U_nu(x-nu)^dagger [U_mu(x-nu) U_nu(x-nu+mu)] U_mu(x)^dagger
  t = mmd(mdm(Unxmn, mm(load_link(U, xmn, mu), load_link(U, xmn_pm, nu))), Umx);
#pragma unroll
  for (int k = 0; k < 9; ++k) Q.e[k] = cadd(Q.e[k], t.e[k]);
  M3 F;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      F.e[i * 3 + j] = cscale(csub(Q.e[i * 3 + j], cconj(Q.e[j * 3 + i])), 0.125);
  return F;
}

// In the chiral basis sigma_{mu nu} = diag(s^l, s^r) with 2x2 blocks
//   s_{kl} = -eps_{klm} sigma_m (both chiralities), s_{k4} = +sigma_k (l), -sigma_k (r).
// Hence C^{hh} = c_sw (i/2) sum_m sigma_m (x) G^h_m with
//   G^h_m = -B_m + s_h E_m,  B = (F_yz, F_zx, F_xy),  E_m = F_{m t},  s_l = +1, s_r = -1.
__global__ void clover_kernel(const double2* __restrict__ U, double2* __restrict__ C, Geom g,
                              double csw) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  long long r = s;
  c[0] = (int)(r % g.L[0]);
  r /= g.L[0];
  c[1] = (int)(r % g.L[1]);
  r /= g.L[1];
  c[2] = (int)(r % g.L[2]);
  c[3] = (int)(r / g.L[2]);
  M3 Bm[3], Em[3];
  Bm[0] = field_strength(U, g, c, s, 1, 2);
  M3 f02 = field_strength(U, g, c, s, 0, 2);
#pragma unroll
  for (int k = 0; k < 9; ++k) Bm[1].e[k] = cscale(f02.e[k], -1.0);
  Bm[2] = field_strength(U, g, c, s, 0, 1);
  for (int m = 0; m < 3; ++m) Em[m] = field_strength(U, g, c, s, m, 3);
  for (int h = 0; h < 2; ++h) {
    const double sh = h == 0 ? 1.0 : -1.0;
    M3 G[3];
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int k = 0; k < 9; ++k)
        G[m].e[k] = make_double2(-Bm[m].e[k].x + sh * Em[m].e[k].x, -Bm[m].e[k].y + sh * Em[m].e[k].y);
    // spin blocks: (0,0) = G_z, (1,1) = -G_z, (0,1) = G_x - i G_y, (1,0) = G_x + i G_y
    double2* out = C + (s * 2 + h) * 36;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            const int k = i * 3 + j;
            double2 v;
            if (a == 0 && b == 0) v = G[2].e[k];
            else if (a == 1 && b == 1) v = cscale(G[2].e[k], -1.0);
            else if (a == 0) v = make_double2(G[0].e[k].x + G[1].e[k].y, G[0].e[k].y - G[1].e[k].x);
            else v = make_double2(G[0].e[k].x - G[1].e[k].y, G[0].e[k].y + G[1].e[k].x);
            // times c_sw (i/2)
            out[(a * 3 + i) * 6 + b * 3 + j] = make_double2(-0.5 * csw * v.y, 0.5 * csw * v.x);
          }
  }
}

// ------------------------------------------------------------------ block reductions
template <int K>
__device__ inline void block_sum(double2 (&v)[K], double2* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      v[k].x += __shfl_xor_sync(0xffffffffu, v[k].x, o);
      v[k].y += __shfl_xor_sync(0xffffffffu, v[k].y, o);
    }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sm[warp * K + k] = v[k];
  __syncthreads();
  if (threadIdx.x < K) {
    double2 t = make_double2(0, 0);
    for (int w = 0; w < nw; ++w) t = cadd(t, sm[w * K + threadIdx.x]);
    sm[32 * K + threadIdx.x] = t;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sm[32 * K + k];
  __syncthreads();
}

// ------------------------------------------------------------------ Gram-Schmidt
// One CTA per aggregate (blk, h).  The aggregate's test vectors (6 Vb x ntv) are processed in
// column blocks of NB = 4: each block is projected against all earlier columns with classical
// Gram-Schmidt (all coefficients from the same vectors), twice, then orthonormalised column by
// column, again classically and twice.  Element n of the aggregate lives in thread n mod T.
// Output row j of R_i^h = conj(q_j).
constexpr int GS_NB = 4;
constexpr int GS_EMAX = 8;

__global__ void __launch_bounds__(256) gs_kernel(const double2* __restrict__ tv, double2* __restrict__ R,
                                                 Geom g, unsigned* err) {
  __shared__ double2 red[32 * 16 + 16];
  __shared__ double2 coef[AMG_MAX_NTV * GS_NB];
  const long long agg = blockIdx.x;
  const long long blk = agg >> 1;
  const int h = (int)(agg & 1);
  const int T = blockDim.x, tid = threadIdx.x, ntv = g.ntv, nagg = g.nagg;
  long long tvoff[GS_EMAX];
  bool valid[GS_EMAX];
#pragma unroll
  for (int e = 0; e < GS_EMAX; ++e) {
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
  double2 w[GS_EMAX][GS_NB];
  for (int j0 = 0; j0 < ntv; j0 += GS_NB) {
    const int nb = min(GS_NB, ntv - j0);
#pragma unroll
    for (int e = 0; e < GS_EMAX; ++e)
#pragma unroll
      for (int c = 0; c < GS_NB; ++c)
        w[e][c] = (valid[e] && c < nb) ? tv[tvoff[e] + j0 + c] : make_double2(0, 0);
    double2 n0[GS_NB];
#pragma unroll
    for (int c = 0; c < GS_NB; ++c) {
      double s = 0;
#pragma unroll
      for (int e = 0; e < GS_EMAX; ++e) s += w[e][c].x * w[e][c].x + w[e][c].y * w[e][c].y;
      n0[c] = make_double2(s, 0);
    }
    block_sum<GS_NB>(n0, red);
    // projection against the earlier column blocks (block classical GS), twice
    for (int pass = 0; pass < 2 && j0 > 0; ++pass) {
      for (int k0 = 0; k0 < j0; k0 += GS_NB) {
        double2 d[GS_NB * GS_NB];
#pragma unroll
        for (int q = 0; q < GS_NB * GS_NB; ++q) d[q] = make_double2(0, 0);
#pragma unroll
        for (int e = 0; e < GS_EMAX; ++e) {
          if (!valid[e]) continue;
          const int n = tid + e * T;
#pragma unroll
          for (int kk = 0; kk < GS_NB; ++kk) {
            const double2 r = Rblk[(long long)(k0 + kk) * nagg + n];  // conj(q_k)
#pragma unroll
            for (int c = 0; c < GS_NB; ++c) cfma(d[kk * GS_NB + c], r, w[e][c]);
          }
        }
        block_sum<GS_NB * GS_NB>(d, red);
        if (tid < GS_NB * GS_NB) coef[k0 * GS_NB + tid] = d[tid];
      }
      __syncthreads();
      for (int k0 = 0; k0 < j0; k0 += GS_NB) {
#pragma unroll
        for (int e = 0; e < GS_EMAX; ++e) {
          if (!valid[e]) continue;
          const int n = tid + e * T;
#pragma unroll
          for (int kk = 0; kk < GS_NB; ++kk) {
            const double2 q = cconj(Rblk[(long long)(k0 + kk) * nagg + n]);
#pragma unroll
            for (int c = 0; c < GS_NB; ++c) {
              const double2 cf = coef[(k0 + kk) * GS_NB + c];
              w[e][c] = csub(w[e][c], cmul(q, cf));
            }
          }
        }
      }
      __syncthreads();
    }
    // orthonormalise inside the block
#pragma unroll
    for (int c = 0; c < GS_NB; ++c) {
      if (c >= nb) break;
      for (int pass = 0; pass < 2 && c > 0; ++pass) {
        double2 d[GS_NB];
#pragma unroll
        for (int cp = 0; cp < GS_NB; ++cp) {
          d[cp] = make_double2(0, 0);
          if (cp < c)
#pragma unroll
            for (int e = 0; e < GS_EMAX; ++e) cfmac(d[cp], w[e][cp], w[e][c]);
        }
        block_sum<GS_NB>(d, red);
#pragma unroll
        for (int e = 0; e < GS_EMAX; ++e)
#pragma unroll
          for (int cp = 0; cp < GS_NB; ++cp)
            if (cp < c) w[e][c] = csub(w[e][c], cmul(w[e][cp], d[cp]));
      }
      double2 nn[1];
      double s = 0;
#pragma unroll
      for (int e = 0; e < GS_EMAX; ++e) s += w[e][c].x * w[e][c].x + w[e][c].y * w[e][c].y;
      nn[0] = make_double2(s, 0);
      block_sum<1>(nn, red);
      const double nrm = sqrt(nn[0].x);
      if (!(nrm > 1e-12 * sqrt(n0[c].x))) {
        if (tid == 0) atomicOr(err, AMG_EBIT_RANK);
      }
      const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
#pragma unroll
      for (int e = 0; e < GS_EMAX; ++e) w[e][c] = cscale(w[e][c], inv);
    }
#pragma unroll
    for (int e = 0; e < GS_EMAX; ++e) {
      if (!valid[e]) continue;
      const int n = tid + e * T;
#pragma unroll
      for (int c = 0; c < GS_NB; ++c)
        if (c < nb) Rblk[(long long)(j0 + c) * nagg + n] = cconj(w[e][c]);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ D_c = R D P assembly
// With (1 - gamma_mu) = u u^dagger, u^dagger = [1, -b_mu] (b_mu the upper-right 2x2 block of
// gamma_mu in the chiral basis), one forward hop x -> x+mu contributes to R_i D P_j
//     -1/2 P(x)^dagger u u^dagger U_mu(x) P(x+mu) = -1/2 A(x)^dagger Bt(x)
// with A = u^dagger P(x) and Bt = u^dagger U_mu(x) P(x+mu), both 6 x 2ntv.  Job mu sums
// A^dagger Bt over the links of block i: links inside the block go to S_mu, links leaving through
// the +mu face to F_mu.  Job 4 sums P(x)^dagger ((4+m0) + C(x)) P(x) with both chiralities
// stacked in the same 6 rows (only the chirality-diagonal quadrants are kept).
// b_mu: -i sigma_x, -i sigma_y, -i sigma_z, 1.
__device__ inline double2 bmat(int mu, int a, int b) {
  if (mu == 0) return (a != b) ? make_double2(0, -1) : make_double2(0, 0);
  if (mu == 1) return (a == 0 && b == 1) ? make_double2(-1, 0) : ((a == 1 && b == 0) ? make_double2(1, 0) : make_double2(0, 0));
  if (mu == 2) return (a == b) ? make_double2(0, a == 0 ? -1 : 1) : make_double2(0, 0);
  return (a == b) ? make_double2(1, 0) : make_double2(0, 0);
}

template <int TA, int TC>
__global__ void __launch_bounds__(256) assemble_kernel(const double2* __restrict__ R, const double2* __restrict__ U,
                                const double2* __restrict__ clov, double2* __restrict__ part, Geom g,
                                double m0, int ncp, int sb_max) {
  extern __shared__ double2 smem[];
  const long long blk = blockIdx.x;
  const int job = blockIdx.y;
  const int nc = g.nc, ntv = g.ntv, nagg = g.nagg, Vb = (int)g.Vb;
  double2* As = smem;                        // [sb][6][ncp]
  double2* Bs = smem + (size_t)sb_max * 6 * ncp;
  const int ntc = ncp / TC, nta = ncp / TA, ntiles = ntc * nta;
  const int tid = threadIdx.x;
  const int ta = tid / ntc, tc = tid % ntc;
  double2 acc0[TA][TC], acc1[TA][TC];
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = 0; j < TC; ++j) acc0[i][j] = acc1[i][j] = make_double2(0, 0);
  // coarse coordinates of this block and stride of direction mu inside a block
  int Xc[4];
  {
    long long r = blk;
    for (int m = 0; m < 4; ++m) {
      Xc[m] = (int)(r % g.Lc[m]);
      r /= g.Lc[m];
    }
  }
  const int mu = job < 4 ? job : 0;
  int stride_mu = 1;
  for (int m = 0; m < mu; ++m) stride_mu *= g.B[m];
  long long blk_fwd;
  {
    int X[4] = {Xc[0], Xc[1], Xc[2], Xc[3]};
    X[mu] = (X[mu] + 1) % g.Lc[mu];
    blk_fwd = ((long long)(X[3] * g.Lc[2] + X[2]) * g.Lc[1] + X[1]) * g.Lc[0] + X[0];
  }
  for (int s0 = 0; s0 < Vb; s0 += sb_max) {
    const int nsb = min(sb_max, Vb - s0);
    for (int pr = tid; pr < sb_max * ncp; pr += blockDim.x) {
      const int sb = pr / ncp, c = pr % ncp;
      double2 A[6], Bt[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) A[k] = Bt[k] = make_double2(0, 0);
      if (sb < nsb && c < nc) {
        const int sl = s0 + sb;
        const long long site = block_site(g, blk, sl);
        const int hc = c / ntv, j = c % ntv;
        const double2* Rc = R + ((blk * 2 + hc) * (long long)ntv + j) * nagg + sl * 6;
        double2 q[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) q[k] = cconj(Rc[k]);
        if (job < 4) {
          // A = u^dagger P(x): l columns keep the l rows, r columns give -b_mu P_r
          if (hc == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) A[k] = q[k];
          } else {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
              for (int col = 0; col < 3; ++col) {
                double2 t = make_double2(0, 0);
#pragma unroll
                for (int b = 0; b < 2; ++b) cfma(t, bmat(mu, a, b), q[b * 3 + col]);
                A[a * 3 + col] = cscale(t, -1.0);
              }
          }
          // neighbour x + mu and its block
          const int lmu = (sl / stride_mu) % g.B[mu];
          const bool face = lmu == g.B[mu] - 1;
          const int sn = face ? sl - (g.B[mu] - 1) * stride_mu : sl + stride_mu;
          const long long bn = face ? blk_fwd : blk;
          const double2* Rn = R + ((bn * 2 + hc) * (long long)ntv + j) * nagg + sn * 6;
          double2 qn[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) qn[k] = cconj(Rn[k]);
          const double2* Ul = U + (site * 4 + mu) * 9;
          double2 z[6];
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int col = 0; col < 3; ++col) {
              double2 t = make_double2(0, 0);
#pragma unroll
              for (int cp = 0; cp < 3; ++cp) cfma(t, Ul[col * 3 + cp], qn[b * 3 + cp]);
              z[b * 3 + col] = t;
            }
          if (hc == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) Bt[k] = z[k];
          } else {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
              for (int col = 0; col < 3; ++col) {
                double2 t = make_double2(0, 0);
#pragma unroll
                for (int b = 0; b < 2; ++b) cfma(t, bmat(mu, a, b), z[b * 3 + col]);
                Bt[a * 3 + col] = cscale(t, -1.0);
              }
          }
        } else {
          const double2* C6 = clov + (site * 2 + hc) * 36;
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            A[k] = q[k];
            double2 t = cscale(q[k], 4.0 + m0);
#pragma unroll
            for (int kp = 0; kp < 6; ++kp) cfma(t, C6[k * 6 + kp], q[kp]);
            Bt[k] = t;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        As[((size_t)sb * 6 + k) * ncp + c] = A[k];
        Bs[((size_t)sb * 6 + k) * ncp + c] = Bt[k];
      }
    }
    __syncthreads();
    if (tid < ntiles) {
      for (int sb = 0; sb < nsb; ++sb) {
        const int sl = s0 + sb;
        const bool face = job < 4 && ((sl / stride_mu) % g.B[mu]) == g.B[mu] - 1;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          double2 av[TA], bv[TC];
#pragma unroll
          for (int i = 0; i < TA; ++i) av[i] = As[((size_t)sb * 6 + k) * ncp + ta * TA + i];
#pragma unroll
          for (int jj = 0; jj < TC; ++jj) bv[jj] = Bs[((size_t)sb * 6 + k) * ncp + tc * TC + jj];
          if (face) {
#pragma unroll
            for (int i = 0; i < TA; ++i)
#pragma unroll
              for (int jj = 0; jj < TC; ++jj) cfmac(acc1[i][jj], av[i], bv[jj]);
          } else {
#pragma unroll
            for (int i = 0; i < TA; ++i)
#pragma unroll
              for (int jj = 0; jj < TC; ++jj) cfmac(acc0[i][jj], av[i], bv[jj]);
          }
        }
      }
    }
    __syncthreads();
  }
  if (tid < ntiles) {
    double2* P0 = part + ((blk * 5 + job) * 2 + 0) * (long long)nc * nc;
    double2* P1 = P0 + (long long)nc * nc;
#pragma unroll
    for (int i = 0; i < TA; ++i)
#pragma unroll
      for (int jj = 0; jj < TC; ++jj) {
        const int a = ta * TA + i, c = tc * TC + jj;
        if (a < nc && c < nc) {
          P0[a * nc + c] = acc0[i][jj];
          P1[a * nc + c] = acc1[i][jj];
        }
      }
  }
}

// D_c blocks from the partial sums:
//   self:  Diag (chirality-diagonal part) - 1/2 sum_mu (S_mu + g5c S_mu^dagger g5c)
//   +mu:   -1/2 F_mu(i)
//   -mu:   g5c (D_c[i-mu][+mu])^dagger g5c            (Eq. dagger)
// where g5c S^dagger g5c accounts for the backward hops inside the block (gamma_5-hermiticity).
__global__ void combine_kernel(const double2* __restrict__ part, const int* __restrict__ nbr,
                               double2* __restrict__ Dc, Geom g) {
  const long long nc = g.nc;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = g.Vc * 9 * nc * nc;
  if (idx >= total) return;
  const int c = (int)(idx % nc);
  const int a = (int)((idx / nc) % nc);
  const int d = (int)((idx / (nc * nc)) % 9);
  const long long i = idx / (9 * nc * nc);
  const double sa = a < g.ntv ? 1.0 : -1.0, sc = c < g.ntv ? 1.0 : -1.0;
  auto P = [&](long long site, int job, int slot) {
    return part + ((site * 5 + job) * 2 + slot) * nc * nc;
  };
  double2 v;
  if (d == 0) {
    v = ((a < g.ntv) == (c < g.ntv)) ? P(i, 4, 0)[a * nc + c] : make_double2(0, 0);
    for (int mu = 0; mu < 4; ++mu) {
      const double2* S = P(i, mu, 0);
      const double2 s1 = S[a * nc + c], s2 = cconj(S[c * nc + a]);
      v.x -= 0.5 * (s1.x + sa * sc * s2.x);
      v.y -= 0.5 * (s1.y + sa * sc * s2.y);
    }
  } else if (d & 1) {
    const int mu = (d - 1) >> 1;
    v = cscale(P(i, mu, 1)[a * nc + c], -0.5);
  } else {
    const int mu = (d - 2) >> 1;
    const long long j = nbr[i * 9 + d];
    v = cscale(cconj(P(j, mu, 1)[c * nc + a]), -0.5 * sa * sc);
  }
  Dc[idx] = v;
}

// D_c to the apply layout At[i][d][col][row] in FP64 / FP32, or FP16 with one FP32 scale per
// (site, direction): s = maxabs / 2^15, stored = value / s rounded to nearest (Sec. 3: half
// precision storage of D_c).
template <int MODE>
__global__ void quantize_dc_kernel(const double2* __restrict__ Dc, void* __restrict__ out,
                                   float* __restrict__ scale, int nc) {
  __shared__ double red[32];
  const long long blk = blockIdx.x;  // (i, d)
  const double2* src = Dc + blk * (long long)nc * nc;
  const int n2 = nc * nc;
  double inv = 1.0;
  float sf = 1.0f;
  if (MODE == 2) {
    double m = 0;
    for (int e = threadIdx.x; e < n2; e += blockDim.x) m = fmax(m, fmax(fabs(src[e].x), fabs(src[e].y)));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
      red[0] = t;
    }
    __syncthreads();
    const double maxabs = red[0];
    sf = maxabs > 0 ? (float)(maxabs / 32768.0) : 1.0f;
    inv = 1.0 / (double)sf;
    if (threadIdx.x == 0) scale[blk] = sf;
  }
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    const int col = e / nc, row = e % nc;
    const double2 v = src[row * nc + col];
    const long long o = blk * (long long)n2 + e;
    if (MODE == 0) {
      ((double2*)out)[o] = v;
    } else if (MODE == 1) {
      ((float2*)out)[o] = make_float2((float)v.x, (float)v.y);
    } else {
      __half2 hv;
      hv.x = __double2half(v.x * inv);
      hv.y = __double2half(v.y * inv);
      ((__half2*)out)[o] = hv;
    }
  }
}

__global__ void r_to_fp32_kernel(const double2* __restrict__ R, float2* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)R[i].x, (float)R[i].y);
}

}  // namespace

// ------------------------------------------------------------------ host driver
static int round_up(int a, int b) { return (a + b - 1) / b * b; }

// The setup's steps; the caller owns the timing events and frees `part` if a step fails.
static amg_status setup_body(amg_coarse* h, const double2* U, const double2* tv, cudaStream_t st, cudaEvent_t (&ev)[5],
                             double2*& part) {
  const Geom& g = h->g;
  AMG_CUDA_TRY(cudaEventRecord(ev[0], st));
  // clover
  {
    const int T = 128;
    const long long nb = (g.V + T - 1) / T;
    clover_kernel<<<(unsigned)nb, T, 0, st>>>(U, h->clover, g, h->p.csw);
    AMG_LAUNCH_CHECK();
  }
  AMG_CUDA_TRY(cudaEventRecord(ev[1], st));
  // Gram-Schmidt, one CTA per aggregate
  amg_status gs_pair = AMG_ERR_UNSUPPORTED;
  if (h->p.setup_arith == AMG_SETUP_F32PAIR) gs_pair = amg_internal_gs_pair(g, tv, h->R64, h->err, st);
  if (gs_pair == AMG_ERR_UNSUPPORTED) {
    int T = round_up(g.nagg < 256 ? g.nagg : 256, 32);
    if ((g.nagg + T - 1) / T > GS_EMAX) return AMG_ERR_UNSUPPORTED;
    gs_kernel<<<(unsigned)(g.Vc * 2), T, 0, st>>>(tv, h->R64, g, h->err);
    AMG_LAUNCH_CHECK();
  } else if (gs_pair != AMG_OK) {
    return gs_pair;
  }
  AMG_CUDA_TRY(cudaEventRecord(ev[2], st));
  // assembly
  const size_t part_elems = (size_t)g.Vc * 5 * 2 * g.nc * g.nc;
  AMG_CUDA_TRY(cudaMallocAsync((void**)&part, part_elems * sizeof(double2), st));
  if (h->p.setup_arith == AMG_SETUP_F32PAIR) {
    AMG_TRY_INTERNAL(amg_internal_assemble_pair(g, h->R64, U, h->clover, part, h->p.m0, h->err, st));
  } else {
    // 2x4 register tiles up to 2 ntv = 40, 4x4 tiles up to 2 ntv = 64; at most 256 threads
    const bool big = g.nc > 40;
    const int TA = big ? 4 : 2, TC = 4;
    const int ncp = round_up(g.nc, 4);
    const int ntiles = (ncp / TA) * (ncp / TC);
    const int T = round_up(ntiles < 128 ? 128 : ntiles, 32);
    if (T > 256) return AMG_ERR_UNSUPPORTED;
    int sb = 8;
    while (sb > 1 && (size_t)sb * 12 * ncp * sizeof(double2) > 96 * 1024) sb >>= 1;
    const size_t sm = (size_t)sb * 12 * ncp * sizeof(double2);
    dim3 grid((unsigned)g.Vc, 5);
    if (big) {
      AMG_CUDA_TRY(cudaFuncSetAttribute(assemble_kernel<4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      assemble_kernel<4, 4><<<grid, T, sm, st>>>(h->R64, U, h->clover, part, g, h->p.m0, ncp, sb);
    } else {
      AMG_CUDA_TRY(cudaFuncSetAttribute(assemble_kernel<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      assemble_kernel<2, 4><<<grid, T, sm, st>>>(h->R64, U, h->clover, part, g, h->p.m0, ncp, sb);
    }
    AMG_LAUNCH_CHECK();
  }
  {
    const long long total = g.Vc * 9LL * g.nc * g.nc;
    combine_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(part, h->nbr, h->Dc64, g);
    AMG_LAUNCH_CHECK();
  }
  AMG_CUDA_TRY(cudaEventRecord(ev[3], st));
  AMG_CUDA_TRY(cudaFreeAsync(part, st));
  part = nullptr;
  // storage precisions
  {
    const unsigned nblk = (unsigned)(g.Vc * 9);
    switch (h->p.link_prec) {
      case AMG_FP64: quantize_dc_kernel<0><<<nblk, 256, 0, st>>>(h->Dc64, h->Dq, nullptr, g.nc); break;
      case AMG_FP32: quantize_dc_kernel<1><<<nblk, 256, 0, st>>>(h->Dc64, h->Dq, nullptr, g.nc); break;
      case AMG_FP16_SCALED: quantize_dc_kernel<2><<<nblk, 256, 0, st>>>(h->Dc64, h->Dq, h->Dscale, g.nc); break;
      default: break;
    }
    AMG_LAUNCH_CHECK();
    if (h->p.r_prec == AMG_FP32) {
      const long long n = g.Vc * 2LL * g.ntv * g.nagg;
      r_to_fp32_kernel<<<1216, 256, 0, st>>>(h->R64, (float2*)h->Rq, n);
      AMG_LAUNCH_CHECK();
    }
    if (h->p.link_prec == AMG_BF16 || h->p.r_prec == AMG_BF16 ||
        ((h->p.link_prec == AMG_FP32 || h->p.link_prec == AMG_FP16_SCALED) && h->p.max_nrhs >= 4)) {
      amg_status s = amg_internal_tc_prepare(h, st);
      if (s != AMG_OK) return s;
    }
  }
  AMG_CUDA_TRY(cudaEventRecord(ev[4], st));
  AMG_CUDA_TRY(cudaEventSynchronize(ev[4]));
  for (int k = 0; k < 4; ++k) cudaEventElapsedTime(&h->setup_ms[k], ev[k], ev[k + 1]);
  unsigned e = 0;
  AMG_CUDA_TRY(cudaMemcpy(&e, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (e & AMG_EBIT_RANK) return AMG_ERR_RANK_DEFICIENT;
  if (e) {
    amg_note_cuda_error(__FILE__, __LINE__, cudaErrorUnknown);
    return AMG_ERR_CUDA;
  }
  return AMG_OK;
}

amg_status amg_internal_setup(amg_coarse* h, const double2* U, const double2* tv, cudaStream_t st) {
  cudaEvent_t ev[5] = {};
  double2* part = nullptr;
  amg_status s = AMG_OK;
  for (int k = 0; k < 5 && s == AMG_OK; ++k) {
    const cudaError_t c = cudaEventCreate(&ev[k]);
    if (c != cudaSuccess) {
      amg_note_cuda_error(__FILE__, __LINE__, c);
      ev[k] = nullptr;
      s = AMG_ERR_CUDA;
    }
  }
  if (s == AMG_OK) s = setup_body(h, U, tv, st, ev, part);
  if (part) cudaFreeAsync(part, st);  // a step failed between the allocation and its release
  for (int k = 0; k < 5; ++k)
    if (ev[k]) cudaEventDestroy(ev[k]);
  return s;
}
