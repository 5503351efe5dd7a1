// Fine-grid part of the two-level method around the coarse-grid correction:
//   D        the Wilson-clover operator (the fine operator whose blocks Eq. cgo restricts),
//   SAP      the domain-decomposition smoother of Alg. 3 (multiplicative Schwarz over two block
//            colours, each block system solved by minimal-residual steps),
//   V-cycle  Alg. 1: the smoother started from the coarse-grid correction of Alg. 2,
//   solve    the outer FGMRES of Sec. 1, right-preconditioned with the V-cycle.
//
// D psi(x) = (4 + m0) psi(x) + C(x) psi(x)
//            - 1/2 sum_mu [(1 - g_mu) U_mu(x) psi(x + mu) + (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)],
// periodic, chiral basis g_mu = [[0, A_mu], [A_mu^dag, 0]] with A = -i sigma_1, -i sigma_2, -i sigma_3, 1.
// Each hop is spin-projected: with psi = (u, d) (spins 0,1 and 2,3),
//   (1 - g) psi = (h, -A^dag h), h = u - A d;   (1 + g) psi = (h', A^dag h'), h' = u + A d,
// so a hop costs two colour mat-vecs (on h) instead of four.  The clover term acts on the two
// chirality halves with the handle's 6x6 blocks C^{ll}, C^{rr}.
//
// The smoother's blocks are the aggregation blocks.  One half sweep (colour c) is one launch: one
// CTA per (block of colour c, right-hand side), one thread per site.  The CTA forms the residual
// r = y - D x on its sites (the neighbours outside the block have the other colour and are not
// written in this launch), runs n_mr MR steps on B e = r with B = D without the hops that cross
// the block face (rho in shared memory, block-wide sums), and adds e to x.
#include "amg_internal.cuh"

#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

namespace {

template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };

template <typename C> __device__ __forceinline__ C zadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C zsub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C zneg(C a) { a.x = -a.x; a.y = -a.y; return a; }
template <typename C> __device__ __forceinline__ C zi(C a) { C r; r.x = -a.y; r.y = a.x; return r; }    // i a
template <typename C> __device__ __forceinline__ C zmi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }   // -i a
template <typename C> __device__ __forceinline__ C zzero() { C r; r.x = 0; r.y = 0; return r; }
template <typename C, typename T> __device__ __forceinline__ C zscale(C a, T s) { a.x *= s; a.y *= s; return a; }
template <typename C> __device__ __forceinline__ void zfma(C& acc, C a, C b) {  // acc += a b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
template <typename C> __device__ __forceinline__ void zfmac(C& acc, C a, C b) {  // acc += conj(a) b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// (A_mu d)_s, s = 0, 1
template <typename C>
__device__ __forceinline__ void amul(int mu, C d0, C d1, C& o0, C& o1) {
  if (mu == 0) { o0 = zmi(d1); o1 = zmi(d0); }          // -i sigma_1
  else if (mu == 1) { o0 = zneg(d1); o1 = d0; }         // -i sigma_2 = [[0, -1], [1, 0]]
  else if (mu == 2) { o0 = zmi(d0); o1 = zi(d1); }      // -i sigma_3
  else { o0 = d0; o1 = d1; }                            // 1
}
// (A_mu^dag v)_s
template <typename C>
__device__ __forceinline__ void adagmul(int mu, C v0, C v1, C& o0, C& o1) {
  if (mu == 0) { o0 = zi(v1); o1 = zi(v0); }            // i sigma_1
  else if (mu == 1) { o0 = v1; o1 = zneg(v0); }         // i sigma_2 = [[0, 1], [-1, 0]]
  else if (mu == 2) { o0 = zi(v0); o1 = zmi(v1); }      // i sigma_3
  else { o0 = v0; o1 = v1; }
}

// out += -1/2 (1 - g_mu) U p   (FWD) or   out += -1/2 (1 + g_mu) U^dag p   (!FWD); p, out: [spin][colour];
// u: the link's 3x3 entries
template <bool FWD, int mu, typename C>
__device__ __forceinline__ void hop_u(const C u[9], const C p[12], C out[12]) {
  C h[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    C a0, a1;
    amul(mu, p[6 + c], p[9 + c], a0, a1);
    h[0][c] = FWD ? zsub(p[c], a0) : zadd(p[c], a0);
    h[1][c] = FWD ? zsub(p[3 + c], a1) : zadd(p[3 + c], a1);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    C w0 = zzero<C>(), w1 = zzero<C>();
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (FWD) {
        zfma(w0, u[a * 3 + b], h[0][b]);
        zfma(w1, u[a * 3 + b], h[1][b]);
      } else {
        zfmac(w0, u[b * 3 + a], h[0][b]);
        zfmac(w1, u[b * 3 + a], h[1][b]);
      }
    }
    C d0, d1;
    adagmul(mu, w0, w1, d0, d1);
    // upper half -1/2 W; lower half +1/2 A^dag W (forward) or -1/2 A^dag W (backward)
    out[a] = zsub(out[a], zscale(w0, 0.5));
    out[3 + a] = zsub(out[3 + a], zscale(w1, 0.5));
    if (FWD) {
      out[6 + a] = zadd(out[6 + a], zscale(d0, 0.5));
      out[9 + a] = zadd(out[9 + a], zscale(d1, 0.5));
    } else {
      out[6 + a] = zsub(out[6 + a], zscale(d0, 0.5));
      out[9 + a] = zsub(out[9 + a], zscale(d1, 0.5));
    }
  }
}

// The 3x3 link at U9 = U + (s 4 + mu) 9.  FP32: 72 bytes from an offset 16-byte aligned for even mu
// and 8 bytes past that for odd mu (s 4 + mu has the parity of mu), so four 16-byte loads and one
// 8-byte load.
template <int mu>
__device__ __forceinline__ void load_link(const double2* __restrict__ U9, double2 u[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = __ldg(U9 + k);
}
template <int mu>
__device__ __forceinline__ void load_link(const float2* __restrict__ U9, float2 u[9]) {
  constexpr int o = mu & 1;  // entries before the first 16-byte boundary
  if (o) u[0] = __ldg(U9);
  const float4* q = reinterpret_cast<const float4*>(U9 + o);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 f = __ldg(q + k);
    u[o + 2 * k] = make_float2(f.x, f.y);
    u[o + 2 * k + 1] = make_float2(f.z, f.w);
  }
  if (!o) u[8] = __ldg(U9 + 8);
}

template <bool FWD, int mu, typename C>
__device__ __forceinline__ void hop(const C* __restrict__ U, const C p[12], C out[12]) {
  C u[9];
  load_link<mu>(U, u);
  hop_u<FWD, mu>(u, p, out);
}

// Row of six clover entries (FP64 blocks)
__device__ __forceinline__ void clover_row(const double2* __restrict__ row, double2 c[6]) {
#pragma unroll
  for (int b = 0; b < 6; ++b) c[b] = __ldg(row + b);
}

// out = (4 + m0) p + C(x) p for the site whose clover blocks start at Cl ([2][6][6])
template <typename C, typename T>
__device__ __forceinline__ void site_term(const C* __restrict__ Cl, T mass, const C p[12], C out[12]) {
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      C acc = zscale(p[hh * 6 + a], mass), c[6];
      clover_row(Cl + (hh * 6 + a) * 6, c);
#pragma unroll
      for (int b = 0; b < 6; ++b) zfma(acc, c[b], p[hh * 6 + b]);
      out[hh * 6 + a] = acc;
    }
  }
}

__host__ __device__ __forceinline__ int tri_index(int a, int b) { return a * 6 - a * (a - 1) / 2 + (b - a); }  // a <= b

// FP32 clover of one site in HBM as the two Hermitian blocks' upper triangles with the diagonal
// (21 entries each in tri_index order, one padding entry after each: 44 complex, 352 bytes instead
// of 576; C_ba = conj(C_ab)), read with 16-byte loads
constexpr int kClPacked = 44;
__device__ __forceinline__ void site_term_hp(const float2* __restrict__ Cl, float mass, const float2 p[12],
                                             float2 out[12]) {
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    float2 c[22];
    const float4* q = reinterpret_cast<const float4*>(Cl + hh * 22);
#pragma unroll
    for (int k = 0; k < 11; ++k) {
      const float4 f = __ldg(q + k);
      c[2 * k] = make_float2(f.x, f.y);
      c[2 * k + 1] = make_float2(f.z, f.w);
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      float2 acc = zscale(p[hh * 6 + a], mass);
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        if (a <= b) zfma(acc, c[tri_index(a, b)], p[hh * 6 + b]);
        else zfmac(acc, c[tri_index(b, a)], p[hh * 6 + b]);
      }
      out[hh * 6 + a] = acc;
    }
  }
}
// the site term of site s: FP32 from the packed clover, FP64 from the full [2][6][6] blocks
template <typename C, typename T>
__device__ __forceinline__ void site_term_at(const C* __restrict__ Cl, long long s, T mass, const C p[12], C out[12]) {
  if constexpr (sizeof(C) == 8) site_term_hp(Cl + s * kClPacked, mass, p, out);
  else site_term(Cl + s * 72, mass, p, out);
}

struct FineGeom {
  int L[4];
  long long V;
  int B[4];
  int Lc[4];
  int Vb;
};

__device__ __forceinline__ void site_coords(const FineGeom& g, long long s, int x[4]) {
  x[0] = (int)(s % g.L[0]);
  s /= g.L[0];
  x[1] = (int)(s % g.L[1]);
  s /= g.L[1];
  x[2] = (int)(s % g.L[2]);
  x[3] = (int)(s / g.L[2]);
}

__device__ __forceinline__ long long site_of(const FineGeom& g, const int x[4]) {
  return (((long long)x[3] * g.L[2] + x[2]) * g.L[1] + x[1]) * g.L[0] + x[0];
}

template <typename C>
__device__ __forceinline__ void load12(const C* __restrict__ v, long long site, int nrhs, int r, C p[12]) {
  if (nrhs == 1 && sizeof(C) == 8) {  // one column of FP32: six 16-byte loads
    const float4* q = reinterpret_cast<const float4*>(v + site * 12);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float4 f = __ldg(q + k);
      p[2 * k].x = f.x;
      p[2 * k].y = f.y;
      p[2 * k + 1].x = f.z;
      p[2 * k + 1].y = f.w;
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) p[k] = v[(site * 12 + k) * nrhs + r];
}

// site +- mu (periodic) from the coordinates of site s
template <int mu, int dir>
__device__ __forceinline__ long long nbr_site(const FineGeom& g, long long s, const int x[4]) {
  long long st = 1;
#pragma unroll
  for (int k = 0; k < mu; ++k) st *= g.L[k];
  if (dir > 0) return x[mu] + 1 < g.L[mu] ? s + st : s - st * (g.L[mu] - 1);
  return x[mu] > 0 ? s - st : s + st * (g.L[mu] - 1);
}

// out += all 8 hops of D at site s (neighbour spinors from v)
template <typename C>
__device__ __forceinline__ void all_hops(const FineGeom& g, const C* __restrict__ U, const C* __restrict__ v,
                                         long long s, const int x[4], int nrhs, int r, C o[12]) {
  C p[12];
#define AMG_HOPS(MU)                                      \
  {                                                       \
    const long long sf = nbr_site<MU, 1>(g, s, x);        \
    load12(v, sf, nrhs, r, p);                            \
    hop<true, MU>(U + (s * 4 + MU) * 9, p, o);            \
    const long long sb = nbr_site<MU, -1>(g, s, x);       \
    load12(v, sb, nrhs, r, p);                            \
    hop<false, MU>(U + (sb * 4 + MU) * 9, p, o);          \
  }
  AMG_HOPS(0)
  AMG_HOPS(1)
  AMG_HOPS(2)
  AMG_HOPS(3)
#undef AMG_HOPS
}

// out = D psi (SUB: out = y - D psi), one thread per (site, right-hand side)
template <typename T, bool SUB>
__global__ void __launch_bounds__(128) dirac_kernel(const typename Cx<T>::type* __restrict__ U,
                                                    const typename Cx<T>::type* __restrict__ Cl,
                                                    const typename Cx<T>::type* __restrict__ psi,
                                                    const typename Cx<T>::type* __restrict__ y,
                                                    typename Cx<T>::type* __restrict__ out, FineGeom g, T mass,
                                                    int nrhs) {
  using C = typename Cx<T>::type;
  const long long total = g.V * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / nrhs;
    const int r = (int)(e % nrhs);
    int x[4];
    site_coords(g, s, x);
    C p[12], o[12];
    load12(psi, s, nrhs, r, p);
    site_term_at(Cl, s, mass, p, o);
    all_hops(g, U, psi, s, x, nrhs, r, o);
    if (SUB) {
      load12(y, s, nrhs, r, p);
#pragma unroll
      for (int k = 0; k < 12; ++k) o[k] = zsub(p[k], o[k]);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) out[(s * 12 + k) * nrhs + r] = o[k];
  }
}

// MR coefficient alpha = <p, rho> / <p, p> from per-thread partial sums v = (<p,p>, Re, Im <p,rho>):
// warp sums, then the CTA sum and the division by one thread, all in the vector precision (FP64
// is slow on this GPU: every thread summing and dividing in FP64 had kept the FP64 pipe busy, and
// one thread's FP64 division held the whole CTA at the barrier), alpha broadcast through shared
// memory.  ok = false when <p, p> = 0.  red: 3 doubles per warp + 3 doubles.
template <typename T, typename C>
__device__ __forceinline__ void cta_alpha(T v[3], double* red, C& al, bool& ok) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  __syncthreads();  // red may still be read by the previous call
  if (lane == 0)
    for (int k = 0; k < 3; ++k) red[warp * 3 + k] = (double)v[k];
  __syncthreads();
  double* out = red + 3 * nw;
  if (threadIdx.x == 0) {
    T sp = 0, sr = 0, si = 0;
    for (int w = 0; w < nw; ++w) {
      sp += (T)red[w * 3];
      sr += (T)red[w * 3 + 1];
      si += (T)red[w * 3 + 2];
    }
    out[0] = sp > 0 ? (double)(sr / sp) : 0.0;
    out[1] = sp > 0 ? (double)(si / sp) : 0.0;
    red[3 * nw + 2] = sp > 0 ? 1.0 : 0.0;
  }
  __syncthreads();
  al.x = (T)out[0];
  al.y = (T)out[1];
  ok = out[2] != 0.0;
}

// The same coefficient with one barrier: each warp's lane 0 writes the warp's partial sums to its
// slot of red (3 values per warp, FP32), and after the barrier every thread sums the slots in warp
// order and divides, so that all threads hold the same alpha (the order and the arithmetic of
// cta_alpha, hence the same value).  Callers alternate between two red buffers from one step to the
// next, so that a step's writes never meet the previous step's reads.
__device__ __forceinline__ void cta_alpha_all(float v[3], float* red, float2& al, bool& ok) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
    for (int k = 0; k < 3; ++k) red[warp * 3 + k] = v[k];
  __syncthreads();
  float sp = 0, sr = 0, si = 0;
  for (int w = 0; w < nw; ++w) {
    sp += red[w * 3];
    sr += red[w * 3 + 1];
    si += red[w * 3 + 2];
  }
  ok = sp > 0;
  al.x = ok ? sr / sp : 0.f;
  al.y = ok ? si / sp : 0.f;
}

// Intra-block hops of the block operator B at local site t: neighbours' rho from shared memory
// (component-major: rho[q * Vb + t]), links from global memory.
template <int mu, typename C>
__device__ __forceinline__ void block_hops_mu(const FineGeom& g, const C* __restrict__ U, const C* rho, int t,
                                              long long s, const int x[4], const int lc[4], int stride, C o[12]) {
  C p[12];
  if (lc[mu] + 1 < g.B[mu]) {
#pragma unroll
    for (int q = 0; q < 12; ++q) p[q] = rho[q * g.Vb + t + stride];
    hop<true, mu>(U + (s * 4 + mu) * 9, p, o);
  }
  if (lc[mu] > 0) {
#pragma unroll
    for (int q = 0; q < 12; ++q) p[q] = rho[q * g.Vb + t - stride];
    const long long sb = nbr_site<mu, -1>(g, s, x);
    hop<false, mu>(U + (sb * 4 + mu) * 9, p, o);
  }
}

// One SAP half sweep on the blocks of one colour: x += MR_{n_mr}(B_b, (y - D x)|_b) per block.
// grid (Vc / 2, nrhs); blockDim >= Vb (threads past Vb only join the sums); dynamic smem: rho
// [12][Vb] + 3 doubles per warp + 3 doubles.
template <typename T>
__global__ void __launch_bounds__(256) sap_kernel(const typename Cx<T>::type* __restrict__ U,
                                                  const typename Cx<T>::type* __restrict__ Cl,
                                                  const typename Cx<T>::type* __restrict__ y,
                                                  typename Cx<T>::type* __restrict__ x, FineGeom g, T mass,
                                                  int nrhs, int colour, int n_mr) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  C* rho = reinterpret_cast<C*>(smem);
  double* red = reinterpret_cast<double*>(smem + (size_t)g.Vb * 12 * sizeof(C));
  const int r = blockIdx.y;
  // the k-th block of this colour: rows of Lc[0] / 2 blocks, X of the colour's parity in each row
  const long long k = blockIdx.x;
  const int half = g.Lc[0] / 2;
  long long row = k / half;
  const int Y = (int)(row % g.Lc[1]);
  row /= g.Lc[1];
  const int Z = (int)(row % g.Lc[2]);
  const int Tt = (int)(row / g.Lc[2]);
  const int X = 2 * (int)(k % half) + ((colour + Y + Z + Tt) & 1);
  const int t = threadIdx.x;
  const bool act = t < g.Vb;
  int lc[4] = {0, 0, 0, 0}, xs[4] = {0, 0, 0, 0};
  long long s = 0;
  if (act) {
    lc[0] = t % g.B[0];
    lc[1] = (t / g.B[0]) % g.B[1];
    lc[2] = (t / (g.B[0] * g.B[1])) % g.B[2];
    lc[3] = t / (g.B[0] * g.B[1] * g.B[2]);
    xs[0] = X * g.B[0] + lc[0];
    xs[1] = Y * g.B[1] + lc[1];
    xs[2] = Z * g.B[2] + lc[2];
    xs[3] = Tt * g.B[3] + lc[3];
    s = site_of(g, xs);
  }
  const int st1 = g.B[0], st2 = g.B[0] * g.B[1], st3 = g.B[0] * g.B[1] * g.B[2];
  // residual r = y - D x on this site (full D: neighbours outside the block have the other colour)
  C o[12], e[12];
  if (act) {
    C p[12];
    load12(x, s, nrhs, r, p);
    site_term_at(Cl, s, mass, p, o);
    all_hops(g, U, x, s, xs, nrhs, r, o);
    load12(y, s, nrhs, r, p);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      rho[q * g.Vb + t] = zsub(p[q], o[q]);
      e[q] = zzero<C>();
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int it = 0; it < n_mr; ++it) {
    // p = B rho at this site: site term plus the hops that stay inside the block
    T v[3] = {0, 0, 0};
    C rr[12];
    if (act) {
#pragma unroll
      for (int q = 0; q < 12; ++q) rr[q] = rho[q * g.Vb + t];
      site_term_at(Cl, s, mass, rr, o);
      block_hops_mu<0>(g, U, rho, t, s, xs, lc, 1, o);
      block_hops_mu<1>(g, U, rho, t, s, xs, lc, st1, o);
      block_hops_mu<2>(g, U, rho, t, s, xs, lc, st2, o);
      block_hops_mu<3>(g, U, rho, t, s, xs, lc, st3, o);
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        v[0] += o[q].x * o[q].x + o[q].y * o[q].y;        // <p, p>
        v[1] += o[q].x * rr[q].x + o[q].y * rr[q].y;      // Re <p, rho>
        v[2] += o[q].x * rr[q].y - o[q].y * rr[q].x;      // Im <p, rho>
      }
    }
    C al;
    bool ok;
    cta_alpha(v, red, al, ok);  // also orders every read of rho before the writes below
    if (act && ok) {
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        zfma(e[q], al, rr[q]);
        C ap = zzero<C>();
        zfma(ap, al, o[q]);
        rho[q * g.Vb + t] = zsub(rr[q], ap);
      }
    }
    __syncthreads();
  }
  if (act) {
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const long long idx = (s * 12 + q) * nrhs + r;
      x[idx] = zadd(x[idx], e[q]);
    }
  }
}

// The same half sweep with the block's links and clover staged in shared memory once, so that
// the MR steps read no global memory (FP32; a 4^4 block takes 74 KB of links, 90 KB of clover and
// 25 KB of rho).  Every staged record keeps its HBM order in pairs of entries, one float4 per pair,
// laid out [pair][Vb]: the threads of a warp (one site each) then read 512 consecutive bytes with
// 16-byte loads, and the staging copies the 16-byte pieces as they lie in HBM (cp.async, no
// register round trip).  Links [18][Vb] (the site's 36 entries, 9 per direction); clover [22][Vb]
// (per chirality the upper triangle with the diagonal, 21 entries padded to 22: the blocks are
// Hermitian, C_ba = conj(C_ab)); rho [6][Vb].
__device__ __forceinline__ float2 lo2(float4 f) { return make_float2(f.x, f.y); }
__device__ __forceinline__ float2 hi2(float4 f) { return make_float2(f.z, f.w); }
// Entry e of a staged record at local site t (the low or high half of pair e / 2)
__device__ __forceinline__ float2 staged_entry(const float4* S, int Vb, int t, int e) {
  return reinterpret_cast<const float2*>(S + (size_t)(e >> 1) * Vb + t)[e & 1];
}
// The link of direction mu at local site t: entries 9 mu .. 9 mu + 8, four pairs and one half
template <int mu>
__device__ __forceinline__ void staged_link(const float4* Us, int Vb, int t, float2 u[9]) {
  constexpr int e0 = 9 * mu, o = e0 & 1, p0 = e0 >> 1;
  if (o) u[0] = staged_entry(Us, Vb, t, e0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 f = Us[(size_t)(p0 + o + k) * Vb + t];
    u[o + 2 * k] = lo2(f);
    u[o + 2 * k + 1] = hi2(f);
  }
  if (!o) u[8] = staged_entry(Us, Vb, t, e0 + 8);
}
__device__ __forceinline__ void staged_spinor(const float4* R, int Vb, int t, float2 p[12]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 f = R[(size_t)k * Vb + t];
    p[2 * k] = lo2(f);
    p[2 * k + 1] = hi2(f);
  }
}
__device__ __forceinline__ void store_spinor(float4* R, int Vb, int t, const float2 p[12]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) R[(size_t)k * Vb + t] = make_float4(p[2 * k].x, p[2 * k].y, p[2 * k + 1].x, p[2 * k + 1].y);
}
// 16-byte global -> shared copy that bypasses the registers (and L1)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void site_term_packed(const float4* Cs, int Vb, int t, float mass, const float2 p[12],
                                                 float2 out[12]) {
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    float2 c[21];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      const float4 f = Cs[(size_t)(hh * 11 + k) * Vb + t];
      c[2 * k] = lo2(f);
      c[2 * k + 1] = hi2(f);
    }
    c[20] = staged_entry(Cs, Vb, t, hh * 22 + 20);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      float2 acc = zscale(p[hh * 6 + a], mass);
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        if (a <= b) zfma(acc, c[tri_index(a, b)], p[hh * 6 + b]);
        else zfmac(acc, c[tri_index(b, a)], p[hh * 6 + b]);
      }
      out[hh * 6 + a] = acc;
    }
  }
}

template <int mu>
__device__ __forceinline__ void block_hops_smem(const float4* Us, const float4* rho, int Vb, int t, const int lc[4],
                                                int bmu, int stride, float2 o[12]) {
  float2 p[12], u[9];
  if (lc[mu] + 1 < bmu) {
    staged_spinor(rho, Vb, t + stride, p);
    staged_link<mu>(Us, Vb, t, u);
    hop_u<true, mu>(u, p, o);
  }
  if (lc[mu] > 0) {
    staged_spinor(rho, Vb, t - stride, p);
    staged_link<mu>(Us, Vb, t - stride, u);
    hop_u<false, mu>(u, p, o);
  }
}

// Both hops of direction mu of the full D at site s (neighbour spinors from global memory), links
// from the staged block where they lie in it: the forward link always, the backward one unless the
// neighbour is outside the block.
template <int mu>
__device__ __forceinline__ void residual_hops(const FineGeom& g, const float2* __restrict__ U, const float4* Us,
                                              const float2* __restrict__ v, long long s, const int x[4], const int lc[4],
                                              int Vb, int t, int stride, int nrhs, int r, float2 o[12]) {
  float2 p[12], u[9];
  load12(v, nbr_site<mu, 1>(g, s, x), nrhs, r, p);
  staged_link<mu>(Us, Vb, t, u);
  hop_u<true, mu>(u, p, o);
  const long long sb = nbr_site<mu, -1>(g, s, x);
  load12(v, sb, nrhs, r, p);
  if (lc[mu] > 0) {
    staged_link<mu>(Us, Vb, t - stride, u);
  } else {
    load_link<mu>(U + (sb * 4 + mu) * 9, u);
  }
  hop_u<false, mu>(u, p, o);
}

__global__ void __launch_bounds__(256, 1) sap_smem_kernel(const float2* __restrict__ U, const float2* __restrict__ Cl,
                                                          const float2* __restrict__ y, float2* __restrict__ x,
                                                          FineGeom g, float mass, int nrhs, int colour, int n_mr) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int Vb = g.Vb;
  float4* Us = reinterpret_cast<float4*>(smem);
  float4* Cs = Us + (size_t)18 * Vb;
  float4* rho = Cs + (size_t)22 * Vb;
  // two buffers of the MR coefficient's warp sums, 3 floats per warp each
  float* redf = reinterpret_cast<float*>(rho + (size_t)6 * Vb);
  const int r = blockIdx.y;
  const long long k = blockIdx.x;
  const int half = g.Lc[0] / 2;
  long long row = k / half;
  const int Y = (int)(row % g.Lc[1]);
  row /= g.Lc[1];
  const int Z = (int)(row % g.Lc[2]);
  const int Tt = (int)(row / g.Lc[2]);
  const int X = 2 * (int)(k % half) + ((colour + Y + Z + Tt) & 1);
  const int t = threadIdx.x;
  const bool act = t < Vb;
  int lc[4] = {0, 0, 0, 0}, xs[4] = {0, 0, 0, 0};
  long long s = 0;
  if (act) {
    lc[0] = t % g.B[0];
    lc[1] = (t / g.B[0]) % g.B[1];
    lc[2] = (t / (g.B[0] * g.B[1])) % g.B[2];
    lc[3] = t / (g.B[0] * g.B[1] * g.B[2]);
    xs[0] = X * g.B[0] + lc[0];
    xs[1] = Y * g.B[1] + lc[1];
    xs[2] = Z * g.B[2] + lc[2];
    xs[3] = Tt * g.B[3] + lc[3];
    s = site_of(g, xs);
  }
  const int st1 = g.B[0], st2 = g.B[0] * g.B[1], st3 = g.B[0] * g.B[1] * g.B[2];
  float2 o[12], e[12];
  if (act) {
    // stage this site's links (288 bytes) and packed clover (352 bytes) as they lie in HBM
    const float4* U4 = reinterpret_cast<const float4*>(U + s * 36);
#pragma unroll
    for (int q = 0; q < 18; ++q) cp_async16(Us + (size_t)q * Vb + t, U4 + q);
    const float4* C4 = reinterpret_cast<const float4*>(Cl + s * kClPacked);
#pragma unroll
    for (int q = 0; q < 22; ++q) cp_async16(Cs + (size_t)q * Vb + t, C4 + q);
  }
  cp_async_wait_all();
  __syncthreads();  // links and clover staged
  if (act) {
    // residual r = y - D x on this site (full D: neighbours outside the block have the other colour);
    // the clover, the forward links and the backward links inside the block from shared memory
    float2 p[12];
    load12(x, s, nrhs, r, p);
    site_term_packed(Cs, Vb, t, mass, p, o);
    residual_hops<0>(g, U, Us, x, s, xs, lc, Vb, t, 1, nrhs, r, o);
    residual_hops<1>(g, U, Us, x, s, xs, lc, Vb, t, st1, nrhs, r, o);
    residual_hops<2>(g, U, Us, x, s, xs, lc, Vb, t, st2, nrhs, r, o);
    residual_hops<3>(g, U, Us, x, s, xs, lc, Vb, t, st3, nrhs, r, o);
    load12(y, s, nrhs, r, p);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      p[q] = zsub(p[q], o[q]);
      e[q] = zzero<float2>();
    }
    store_spinor(rho, Vb, t, p);
  }
  __syncthreads();
#pragma unroll 1
  for (int it = 0; it < n_mr; ++it) {
    // p = B rho at this site: site term plus the hops that stay inside the block
    float v[3] = {0, 0, 0};
    float2 rr[12];
    if (act) {
      staged_spinor(rho, Vb, t, rr);
      site_term_packed(Cs, Vb, t, mass, rr, o);
      block_hops_smem<0>(Us, rho, Vb, t, lc, g.B[0], 1, o);
      block_hops_smem<1>(Us, rho, Vb, t, lc, g.B[1], st1, o);
      block_hops_smem<2>(Us, rho, Vb, t, lc, g.B[2], st2, o);
      block_hops_smem<3>(Us, rho, Vb, t, lc, g.B[3], st3, o);
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        v[0] += o[q].x * o[q].x + o[q].y * o[q].y;        // <p, p>
        v[1] += o[q].x * rr[q].x + o[q].y * rr[q].y;      // Re <p, rho>
        v[2] += o[q].x * rr[q].y - o[q].y * rr[q].x;      // Im <p, rho>
      }
    }
    float2 al;
    bool ok;
    // also orders every read of rho before the writes below
    cta_alpha_all(v, redf + (it & 1) * 3 * ((blockDim.x + 31) >> 5), al, ok);
    if (act && ok) {
      float2 nr[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        zfma(e[q], al, rr[q]);
        float2 ap = zzero<float2>();
        zfma(ap, al, o[q]);
        nr[q] = zsub(rr[q], ap);
      }
      store_spinor(rho, Vb, t, nr);
    }
    __syncthreads();
  }
  if (act) {
    if (nrhs == 1) {  // one column: the site's 96 bytes as six 16-byte words
      float4* x4 = reinterpret_cast<float4*>(x + s * 12);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        float4 f = x4[k];
        f.x += e[2 * k].x;
        f.y += e[2 * k].y;
        f.z += e[2 * k + 1].x;
        f.w += e[2 * k + 1].y;
        x4[k] = f;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const long long idx = (s * 12 + q) * nrhs + r;
        x[idx] = zadd(x[idx], e[q]);
      }
    }
  }
}

// ------------------------------------------------------------------ outer FGMRES vector kernels
constexpr int FT = 256;

// Arithmetic of the outer FGMRES vector kernels: per element in the vectors' precision (FP64 is
// slow on this GPU; an FP32 vector gains nothing from FP64 products), per-thread partial sums in
// that precision (a few dozen elements each), sums across threads and CTAs in FP64.  The per-column
// coefficients are converted to the vectors' precision once per CTA, in shared memory.
template <typename C> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

template <typename C>
__device__ __forceinline__ C to_c(double2 v) {
  C o;
  o.x = (typename Real<C>::type)v.x;
  o.y = (typename Real<C>::type)v.y;
  return o;
}

// part[i][r] += sum_n conj(V_i[n, r]) w[n, r] for i < nv (one FP64 atomic per CTA and pair)
template <typename C>
__global__ void __launch_bounds__(FT) fdots_kernel(const C* __restrict__ Vb, long long vstride, int nv,
                                                   const C* __restrict__ w, long long n, int nrhs, double2* out) {
  using R = typename Real<C>::type;
  __shared__ double2 red[FT];
  const int i = blockIdx.y;
  const C* v = Vb + vstride * i;
  const int per = FT / nrhs * nrhs;  // threads per CTA that take part (a multiple of nrhs)
  R ax = 0, ay = 0;
  if (threadIdx.x < per) {
    for (long long e = blockIdx.x * (long long)per + threadIdx.x; e < n * nrhs; e += (long long)gridDim.x * per) {
      const C a = v[e], b = w[e];
      ax = fma(a.x, b.x, fma(a.y, b.y, ax));
      ay = fma(a.x, b.y, fma(-a.y, b.x, ay));
    }
  }
  red[threadIdx.x] = make_double2((double)ax, (double)ay);
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double2 s = make_double2(0, 0);
    for (int q = threadIdx.x; q < per; q += nrhs) {
      s.x += red[q].x;
      s.y += red[q].y;
    }
    atomicAdd(&out[i * nrhs + threadIdx.x].x, s.x);
    atomicAdd(&out[i * nrhs + threadIdx.x].y, s.y);
  }
}

constexpr int kFMaxCoef = 1024;  // coefficients cached per CTA (nv x nrhs); more are read from global memory

template <typename C>
__device__ __forceinline__ C coef_at(const C* cached, const double2* __restrict__ g, bool use_cache, int k) {
  return use_cache ? cached[k] : to_c<C>(g[k]);
}

// w -= sum_{i < nv} h[i][r] V_i ; nrm2[r] += |w|^2 (after the update)
template <typename C>
__global__ void __launch_bounds__(FT) fupdate_kernel(const C* __restrict__ Vb, long long vstride, int nv,
                                                     const double2* __restrict__ h, C* __restrict__ w, long long n,
                                                     int nrhs, double* nrm2) {
  using R = typename Real<C>::type;
  __shared__ double red[FT];
  __shared__ C hc[kFMaxCoef];
  const bool cached = nv * nrhs <= kFMaxCoef;
  if (cached)
    for (int k = threadIdx.x; k < nv * nrhs; k += blockDim.x) hc[k] = to_c<C>(h[k]);
  __syncthreads();
  const int per = FT / nrhs * nrhs;
  R acc = 0;
  if (threadIdx.x < per) {
    for (long long e = blockIdx.x * (long long)per + threadIdx.x; e < n * nrhs; e += (long long)gridDim.x * per) {
      const int r = (int)(e % nrhs);
      C a = w[e];
      for (int i = 0; i < nv; ++i) {
        const C v = Vb[vstride * i + e];
        const C c = coef_at(hc, h, cached, i * nrhs + r);
        a.x -= c.x * v.x - c.y * v.y;
        a.y -= c.x * v.y + c.y * v.x;
      }
      w[e] = a;
      acc = fma(a.x, a.x, fma(a.y, a.y, acc));
    }
  }
  red[threadIdx.x] = (double)acc;
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double s = 0;
    for (int q = threadIdx.x; q < per; q += nrhs) s += red[q];
    atomicAdd(&nrm2[threadIdx.x], s);
  }
}

// y = a[r] * x (a per column, complex); y may be x
template <typename C>
__global__ void fscale_kernel(const C* x, C* y, const double2* __restrict__ a, long long n, int nrhs) {
  __shared__ C ac[64];  // nrhs <= 64
  if (threadIdx.x < nrhs) ac[threadIdx.x] = to_c<C>(a[threadIdx.x]);
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * nrhs;
       e += (long long)gridDim.x * blockDim.x) {
    const C c = ac[e % nrhs];
    const C v = x[e];
    C o;
    o.x = c.x * v.x - c.y * v.y;
    o.y = c.x * v.y + c.y * v.x;
    y[e] = o;
  }
}

// y += sum_{i < nv} c[i][r] X_i
template <typename C>
__global__ void fcombine_kernel(const C* __restrict__ Xb, long long vstride, int nv, const double2* __restrict__ c,
                                C* __restrict__ y, long long n, int nrhs) {
  __shared__ C cc[kFMaxCoef];
  const bool cached = nv * nrhs <= kFMaxCoef;
  if (cached)
    for (int k = threadIdx.x; k < nv * nrhs; k += blockDim.x) cc[k] = to_c<C>(c[k]);
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * nrhs;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % nrhs);
    C a = y[e];
    for (int i = 0; i < nv; ++i) {
      const C v = Xb[vstride * i + e];
      const C k = coef_at(cc, c, cached, i * nrhs + r);
      a.x += k.x * v.x - k.y * v.y;
      a.y += k.x * v.y + k.y * v.x;
    }
    y[e] = a;
  }
}

// nrm2[r] += |v|^2
template <typename C>
__global__ void __launch_bounds__(FT) fnorm_kernel(const C* __restrict__ v, long long n, int nrhs, double* nrm2) {
  using R = typename Real<C>::type;
  __shared__ double red[FT];
  const int per = FT / nrhs * nrhs;
  R acc = 0;
  if (threadIdx.x < per)
    for (long long e = blockIdx.x * (long long)per + threadIdx.x; e < n * nrhs; e += (long long)gridDim.x * per)
      acc = fma(v[e].x, v[e].x, fma(v[e].y, v[e].y, acc));
  red[threadIdx.x] = (double)acc;
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double s = 0;
    for (int q = threadIdx.x; q < per; q += nrhs) s += red[q];
    atomicAdd(&nrm2[threadIdx.x], s);
  }
}

FineGeom fine_geom(const amg_coarse* h) {
  FineGeom g;
  for (int mu = 0; mu < 4; ++mu) {
    g.L[mu] = h->g.L[mu];
    g.B[mu] = h->g.B[mu];
    g.Lc[mu] = h->g.Lc[mu];
  }
  g.V = h->g.V;
  g.Vb = (int)h->g.Vb;
  return g;
}

// FP64 clover blocks [V][2][6][6] -> FP32 packed upper triangles [V][2][22] (tri_index order, the last
// entry of each chirality zero)
__global__ void clover_pack_kernel(const double2* __restrict__ in, float2* __restrict__ out, long long V) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < V * 44; e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / 44;
    const int hh = (int)(e % 44) / 22, k = (int)(e % 22);
    float2 v = make_float2(0.f, 0.f);
    if (k < 21) {
      int a = 0;
      while (tri_index(a, 5) < k) ++a;  // row of entry k: the first row whose last entry is >= k
      const int b = a + (k - tri_index(a, a));
      const double2 d = in[(s * 2 + hh) * 36 + a * 6 + b];
      v = make_float2((float)d.x, (float)d.y);
    }
    out[e] = v;
  }
}

template <typename T>
__global__ void to_prec_kernel(const double2* __restrict__ in, typename Cx<T>::type* __restrict__ out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    typename Cx<T>::type v;
    v.x = (T)in[e].x;
    v.y = (T)in[e].y;
    out[e] = v;
  }
}

bool fine_fp64(const amg_coarse* h) { return h->p.vec_prec == AMG_FP64; }

template <typename T>
amg_status launch_dirac(amg_coarse* h, const void* psi, const void* y, void* out, int nrhs, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const long long total = h->g.V * nrhs;
  const long long want = (total + 127) / 128;
  const int grid = (int)(want < 16LL * amg_sm_count() ? want : 16LL * amg_sm_count());
  const T mass = (T)(4.0 + h->p.m0);
  if (y)
    dirac_kernel<T, true><<<grid, 128, 0, st>>>((const C*)h->fU, (const C*)h->fC, (const C*)psi, (const C*)y, (C*)out,
                                                 fine_geom(h), mass, nrhs);
  else
    dirac_kernel<T, false><<<grid, 128, 0, st>>>((const C*)h->fU, (const C*)h->fC, (const C*)psi, nullptr, (C*)out,
                                                  fine_geom(h), mass, nrhs);
  AMG_LAUNCH_CHECK();
  h->launches++;
  return AMG_OK;
}

amg_status dirac_any(amg_coarse* h, const void* psi, const void* y, void* out, int nrhs, cudaStream_t st) {
  return fine_fp64(h) ? launch_dirac<double>(h, psi, y, out, nrhs, st) : launch_dirac<float>(h, psi, y, out, nrhs, st);
}

template <typename T>
amg_status launch_sap(amg_coarse* h, const void* y, void* x, int nrhs, int n_cycles, int n_mr, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const int threads = (h->g.Vb + 31) / 32 * 32;
  if (sizeof(T) == 4) {
    // links, clover and rho of a block, then two buffers of the MR coefficient's warp sums
    const size_t sm2 = (size_t)h->g.Vb * (18 + 22 + 6) * sizeof(float4) + (size_t)(threads / 32) * 2 * 3 * sizeof(float);
    if (threads <= 256 && sm2 <= 227 * 1024) {
      AMG_CUDA_TRY(cudaFuncSetAttribute(sap_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
      const dim3 grid((unsigned)(h->g.Vc / 2), (unsigned)nrhs);
      const float mass = (float)(4.0 + h->p.m0);
      for (int c = 0; c < n_cycles; ++c)
        for (int colour = 0; colour < 2; ++colour) {
          sap_smem_kernel<<<grid, threads, sm2, st>>>((const float2*)h->fU, (const float2*)h->fC, (const float2*)y,
                                                      (float2*)x, fine_geom(h), mass, nrhs, colour, n_mr);
          AMG_LAUNCH_CHECK();
          h->launches++;
        }
      return AMG_OK;
    }
  }
  const size_t smem = (size_t)h->g.Vb * 12 * sizeof(C) + (size_t)(threads / 32 + 1) * 3 * sizeof(double);
  if (threads > 256 || smem > 227 * 1024) return AMG_ERR_UNSUPPORTED;
  AMG_CUDA_TRY(cudaFuncSetAttribute(sap_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const dim3 grid((unsigned)(h->g.Vc / 2), (unsigned)nrhs);
  const T mass = (T)(4.0 + h->p.m0);
  for (int c = 0; c < n_cycles; ++c)
    for (int colour = 0; colour < 2; ++colour) {
      sap_kernel<T><<<grid, threads, smem, st>>>((const C*)h->fU, (const C*)h->fC, (const C*)y, (C*)x, fine_geom(h),
                                                 mass, nrhs, colour, n_mr);
      AMG_LAUNCH_CHECK();
      h->launches++;
    }
  return AMG_OK;
}

amg_status sap_any(amg_coarse* h, const void* y, void* x, int nrhs, int n_cycles, int n_mr, cudaStream_t st) {
  return fine_fp64(h) ? launch_sap<double>(h, y, x, nrhs, n_cycles, n_mr, st)
                      : launch_sap<float>(h, y, x, nrhs, n_cycles, n_mr, st);
}

amg_status check_fine(amg_coarse* h, const void* a, const void* b, int nrhs) {
  if (!h || !a || !b || !aligned16(a) || !aligned16(b)) return AMG_ERR_INVALID_ARG;
  if (nrhs < 1 || nrhs > h->p.max_nrhs) return AMG_ERR_INVALID_ARG;
  if (!h->fU) return AMG_ERR_UNSUPPORTED;  // amg_setup_fine not called
  return AMG_OK;
}

bool sap_supported(const amg_coarse* h) {
  for (int mu = 0; mu < 4; ++mu)
    if (h->g.Lc[mu] % 2) return false;
  return h->g.Vb <= 256;
}

amg_status check_vp(const amg_vcycle_params* vp) {
  if (!vp || !(vp->coarse_tol >= 0) || vp->coarse_restart < 1 || vp->coarse_max_applies < 1 || vp->n_smoother < 0 ||
      vp->n_mr < 1)
    return AMG_ERR_INVALID_ARG;
  return AMG_OK;
}

amg_status vcycle_impl(amg_coarse* h, const amg_vcycle_params* vp, const void* y, void* x, int nrhs,
                       cudaStream_t st) {
  if (h->next)  // three levels: one two-grid cycle on level 1 in place of the coarse solve
    AMG_TRY_INTERNAL(amg_internal_cgc3(h, y, x, nrhs, st));
  else
    AMG_TRY_INTERNAL(amg_cgc(h, y, x, nrhs, vp->coarse_tol, vp->coarse_restart, vp->coarse_max_applies, st, nullptr));
  if (vp->n_smoother > 0) AMG_TRY_INTERNAL(sap_any(h, y, x, nrhs, vp->n_smoother, vp->n_mr, st));
  return AMG_OK;
}

// ------------------------------------------------------------------ outer FGMRES (host-driven)
// Right-preconditioned flexible GMRES(m) of Saad Alg. 9.6 from u = 0, every right-hand side
// independently: classical Gram-Schmidt Arnoldi, Givens rotations, convergence on the implicit
// residual |g_{j+1}| <= tol ||f||; every restart after the first recomputes the true residual
// (one more application of D), as the coarse solve counts them.  Scalars live on the host: each
// Arnoldi step synchronises once, which is small against the V-cycle it waits for.
template <typename T>
amg_status solve_impl(amg_coarse* h, const amg_vcycle_params* vp, const void* f, void* u, int nrhs, double tol,
                      int m, int max_applies, cudaStream_t st, double* info) {
  using C = typename Cx<T>::type;
  const long long n = h->g.V * 12;
  const long long vs = n * nrhs;  // elements of one multi-column vector
  const size_t vbytes = (size_t)vs * sizeof(C);
  // workspace: V_0..V_m, Z_0..Z_{m-1}, r, and (m + 1) x nrhs double2 + nrhs doubles of sums
  const size_t need = (size_t)(2 * m + 2) * vbytes + ((size_t)(m + 1) * nrhs * 2 + nrhs) * sizeof(double) + 256;
  if (need > h->fwork_bytes) {
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(h->fwork);
    h->fwork = nullptr;
    h->fwork_bytes = 0;
    AMG_CUDA_TRY(cudaMalloc(&h->fwork, need));
    h->fwork_bytes = need;
  }
  C* Vb = (C*)h->fwork;
  C* Zb = Vb + (size_t)(m + 1) * vs;
  C* R = Zb + (size_t)m * vs;
  double2* dh = (double2*)(R + vs);
  double* dn = (double*)(dh + (size_t)(m + 1) * nrhs);
  C* U = (C*)u;
  const int vgrid = 4 * amg_sm_count();
  const dim3 fblk(FT);

  auto colnorm = [&](const C* v, std::vector<double>& out) -> amg_status {
    AMG_CUDA_TRY(cudaMemsetAsync(dn, 0, nrhs * sizeof(double), st));
    fnorm_kernel<C><<<vgrid, fblk, 0, st>>>(v, n, nrhs, dn);
    AMG_LAUNCH_CHECK();
    h->launches++;
    AMG_CUDA_TRY(cudaMemcpyAsync(out.data(), dn, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    for (auto& x : out) x = sqrt(x);
    return AMG_OK;
  };

  std::vector<double> fnorm(nrhs), beta(nrhs), tmp(nrhs);
  std::vector<int> applies(nrhs, 0), done(nrhs, 0);
  std::vector<double> relres(nrhs, 1.0);
  AMG_CUDA_TRY(cudaMemsetAsync(U, 0, vbytes, st));
  AMG_CUDA_TRY(cudaMemcpyAsync(R, f, vbytes, cudaMemcpyDeviceToDevice, st));
  AMG_TRY_INTERNAL(colnorm((const C*)f, fnorm));
  for (int r = 0; r < nrhs; ++r)
    if (fnorm[r] == 0) {
      done[r] = 1;
      relres[r] = 0;
    }
  int total_applies = 0;
  const size_t hs = (size_t)(m + 1) * m;
  std::vector<std::complex<double>> H(hs * nrhs), cs(m * nrhs), sn(m * nrhs), g((m + 1) * nrhs);
  std::vector<double2> coef((m + 1) * nrhs);
  while (true) {
    AMG_TRY_INTERNAL(colnorm(R, beta));
    bool any = false;
    for (int r = 0; r < nrhs; ++r) {
      if (!done[r] && beta[r] <= tol * fnorm[r]) done[r] = 1;
      any = any || !done[r];
    }
    const int mm = std::min(m, max_applies - total_applies);
    if (!any || mm <= 0) break;
    // V_0 = r / beta (columns already converged get 0 and stay 0)
    for (int r = 0; r < nrhs; ++r) coef[r] = make_double2(done[r] ? 0.0 : 1.0 / beta[r], 0.0);
    AMG_CUDA_TRY(cudaMemcpyAsync(dh, coef.data(), nrhs * sizeof(double2), cudaMemcpyHostToDevice, st));
    fscale_kernel<C><<<vgrid, fblk, 0, st>>>(R, Vb, dh, n, nrhs);
    AMG_LAUNCH_CHECK();
    h->launches++;
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    for (int r = 0; r < nrhs; ++r) g[r * (m + 1)] = beta[r];
    std::vector<int> k(nrhs, 0), active(nrhs);
    for (int r = 0; r < nrhs; ++r) active[r] = !done[r];
    for (int j = 0; j < mm; ++j) {
      C* Vj = Vb + (size_t)j * vs;
      C* Zj = Zb + (size_t)j * vs;
      C* W = Vb + (size_t)(j + 1) * vs;
      AMG_TRY_INTERNAL(vcycle_impl(h, vp, Vj, Zj, nrhs, st));        // Z_j = M V_j
      AMG_TRY_INTERNAL(dirac_any(h, Zj, nullptr, W, nrhs, st));      // w = D Z_j
      total_applies++;
      AMG_CUDA_TRY(cudaMemsetAsync(dh, 0, (size_t)(j + 1) * nrhs * sizeof(double2), st));
      fdots_kernel<C><<<dim3(vgrid, j + 1), fblk, 0, st>>>(Vb, vs, j + 1, W, n, nrhs, dh);
      AMG_LAUNCH_CHECK();
      AMG_CUDA_TRY(cudaMemsetAsync(dn, 0, nrhs * sizeof(double), st));
      fupdate_kernel<C><<<vgrid, fblk, 0, st>>>(Vb, vs, j + 1, dh, W, n, nrhs, dn);
      AMG_LAUNCH_CHECK();
      h->launches += 2;
      std::vector<double2> hc((size_t)(j + 1) * nrhs);
      AMG_CUDA_TRY(cudaMemcpyAsync(hc.data(), dh, hc.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
      AMG_CUDA_TRY(cudaMemcpyAsync(tmp.data(), dn, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
      AMG_CUDA_TRY(cudaStreamSynchronize(st));
      bool more = false;
      for (int r = 0; r < nrhs; ++r) {
        coef[r] = make_double2(0, 0);
        if (!active[r]) continue;
        applies[r]++;
        std::complex<double>* Hr = H.data() + hs * r;  // Hr[i * m + j]
        for (int i = 0; i <= j; ++i) Hr[i * m + j] = std::complex<double>(hc[i * nrhs + r].x, hc[i * nrhs + r].y);
        const double hnext = sqrt(tmp[r]);
        Hr[(j + 1) * m + j] = hnext;
        std::complex<double>* c = cs.data() + (size_t)m * r;
        std::complex<double>* s = sn.data() + (size_t)m * r;
        std::complex<double>* gr = g.data() + (size_t)(m + 1) * r;
        for (int i = 0; i < j; ++i) {
          const std::complex<double> a = c[i] * Hr[i * m + j] + s[i] * Hr[(i + 1) * m + j];
          Hr[(i + 1) * m + j] = -std::conj(s[i]) * Hr[i * m + j] + std::conj(c[i]) * Hr[(i + 1) * m + j];
          Hr[i * m + j] = a;
        }
        const std::complex<double> a = Hr[j * m + j], b = Hr[(j + 1) * m + j];
        const double den = sqrt(std::norm(a) + std::norm(b));
        c[j] = std::conj(a) / den;
        s[j] = std::conj(b) / den;
        Hr[j * m + j] = den;
        Hr[(j + 1) * m + j] = 0.0;
        gr[j + 1] = -std::conj(s[j]) * gr[j];
        gr[j] = c[j] * gr[j];
        k[r] = j + 1;
        relres[r] = std::abs(gr[j + 1]) / fnorm[r];
        if (std::abs(gr[j + 1]) <= tol * fnorm[r] || hnext == 0) {
          active[r] = 0;
          done[r] = 1;
        } else {
          coef[r] = make_double2(1.0 / hnext, 0.0);
          more = true;
        }
      }
      if (!more) break;
      // V_{j+1} = w / h_{j+1,j} (columns that stopped get 0 and drop out of later sums)
      AMG_CUDA_TRY(cudaMemcpyAsync(dh, coef.data(), nrhs * sizeof(double2), cudaMemcpyHostToDevice, st));
      AMG_CUDA_TRY(cudaStreamSynchronize(st));
      fscale_kernel<C><<<vgrid, fblk, 0, st>>>(W, W, dh, n, nrhs);
      AMG_LAUNCH_CHECK();
      h->launches++;
    }
    // u += Z y, y from the k x k triangular systems
    std::vector<double2> yv((size_t)m * nrhs, make_double2(0, 0));
    int kmax = 0;
    for (int r = 0; r < nrhs; ++r) {
      const std::complex<double>* Hr = H.data() + hs * r;
      const std::complex<double>* gr = g.data() + (size_t)(m + 1) * r;
      std::vector<std::complex<double>> yy(k[r]);
      for (int i = k[r] - 1; i >= 0; --i) {
        std::complex<double> acc = gr[i];
        for (int q = i + 1; q < k[r]; ++q) acc -= Hr[i * m + q] * yy[q];
        yy[i] = acc / Hr[i * m + i];
      }
      for (int i = 0; i < k[r]; ++i) yv[i * nrhs + r] = make_double2(yy[i].real(), yy[i].imag());
      kmax = std::max(kmax, k[r]);
    }
    if (kmax > 0) {
      AMG_CUDA_TRY(cudaMemcpyAsync(dh, yv.data(), (size_t)kmax * nrhs * sizeof(double2), cudaMemcpyHostToDevice, st));
      fcombine_kernel<C><<<vgrid, fblk, 0, st>>>(Zb, vs, kmax, dh, U, n, nrhs);
      AMG_LAUNCH_CHECK();
      h->launches++;
    }
    bool all = true;
    for (int r = 0; r < nrhs; ++r) all = all && done[r];
    if (all || total_applies >= max_applies) break;
    // true residual r = f - D u
    AMG_TRY_INTERNAL(dirac_any(h, u, f, R, nrhs, st));
    total_applies++;
    for (int r = 0; r < nrhs; ++r)
      if (!done[r]) applies[r]++;
  }
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  if (info)
    for (int r = 0; r < nrhs; ++r) {
      info[2 * r] = applies[r];
      info[2 * r + 1] = relres[r];
    }
  return AMG_OK;
}

// Columns j0 .. j0 + nc - 1 of the FP64 test vectors tv ([V][12][ntv]) <-> a fine vector of nc
// columns in the vector precision ([V][12][nc]).
template <typename C>
__global__ void tv_gather_kernel(const double2* __restrict__ tv, C* __restrict__ out, long long n12, int ntv, int j0,
                                 int nc) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n12 * nc;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 v = tv[(e / nc) * ntv + j0 + (int)(e % nc)];
    C o;
    o.x = v.x;
    o.y = v.y;
    out[e] = o;
  }
}

template <typename C>
__global__ void tv_scatter_kernel(const C* __restrict__ in, double2* __restrict__ tv, long long n12, int ntv, int j0,
                                  int nc) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n12 * nc;
       e += (long long)gridDim.x * blockDim.x)
    tv[(e / nc) * ntv + j0 + (int)(e % nc)] = make_double2((double)in[e].x, (double)in[e].y);
}

// Alg. 4 on the handle: see amg_adaptive_setup in amg.h.  The test vectors go through the smoother
// and the V-cycle in column chunks of at most min(max_nrhs, 16); R and D_c are rebuilt in place.
template <typename T>
amg_status adaptive_impl(amg_coarse* h, const amg_vcycle_params* vp, const double2* U, double2* tv, int n_setup,
                         cudaStream_t st) {
  using C = typename Cx<T>::type;
  const int ntv = h->g.ntv;
  const int chunk = std::min(h->p.max_nrhs, 16);
  const long long n12 = h->g.V * 12;
  const size_t vbytes = (size_t)n12 * chunk * sizeof(C);
  void* buf = nullptr;
  AMG_CUDA_TRY(cudaMallocAsync(&buf, 2 * vbytes + 256 + (size_t)ntv * (sizeof(double) + sizeof(double2)), st));
  C* y = (C*)buf;
  C* x = y + (size_t)n12 * chunk;
  double* dn = (double*)(x + (size_t)n12 * chunk);
  double2* dc = (double2*)(dn + ntv);
  const int vgrid = 4 * amg_sm_count();
  amg_status s = AMG_OK;
  auto each_chunk = [&](auto&& body) -> amg_status {
    for (int j0 = 0; j0 < ntv; j0 += chunk) {
      const int nc = std::min(chunk, ntv - j0);
      tv_gather_kernel<C><<<vgrid, 256, 0, st>>>(tv, y, n12, ntv, j0, nc);
      AMG_LAUNCH_CHECK();
      AMG_TRY_INTERNAL(body(nc));
      tv_scatter_kernel<C><<<vgrid, 256, 0, st>>>(x, tv, n12, ntv, j0, nc);
      AMG_LAUNCH_CHECK();
      h->launches += 2;
    }
    return AMG_OK;
  };
  // initial phase: v <- S_k(v; 0), k = 1, 2, 3
  s = each_chunk([&](int nc) -> amg_status {
    for (int k = 1; k <= 3; ++k) {
      AMG_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)n12 * nc * sizeof(C), st));
      AMG_TRY_INTERNAL(sap_any(h, y, x, nc, k, vp->n_mr, st));
      if (k < 3) AMG_CUDA_TRY(cudaMemcpyAsync(y, x, (size_t)n12 * nc * sizeof(C), cudaMemcpyDeviceToDevice, st));
    }
    return AMG_OK;
  });
  if (s == AMG_OK) s = amg_internal_rebuild(h, U, tv, st);
  if (s == AMG_OK) {  // v_j <- v_j / ||v_j||
    cudaMemsetAsync(dn, 0, ntv * sizeof(double), st);
    fnorm_kernel<double2><<<vgrid, FT, 0, st>>>(tv, n12, ntv, dn);
    std::vector<double> nrm(ntv);
    cudaMemcpyAsync(nrm.data(), dn, ntv * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) s = AMG_ERR_CUDA;
    std::vector<double2> inv(ntv);
    for (int j = 0; j < ntv; ++j) inv[j] = make_double2(nrm[j] > 0 ? 1.0 / sqrt(nrm[j]) : 0.0, 0.0);
    if (s == AMG_OK && cudaMemcpyAsync(dc, inv.data(), ntv * sizeof(double2), cudaMemcpyHostToDevice, st) != cudaSuccess)
      s = AMG_ERR_CUDA;
    if (s == AMG_OK) {
      fscale_kernel<double2><<<vgrid, 256, 0, st>>>(tv, tv, dc, n12, ntv);
      if (cudaGetLastError() != cudaSuccess) s = AMG_ERR_CUDA;
      h->launches += 2;
    }
  }
  // iterative passes: v_j <- S(v_j; CGC(v_j)) with the current R and D_c, then rebuild
  for (int pass = 0; pass < n_setup && s == AMG_OK; ++pass) {
    s = each_chunk([&](int nc) -> amg_status { return vcycle_impl(h, vp, y, x, nc, st); });
    if (s == AMG_OK) s = amg_internal_rebuild(h, U, tv, st);
  }
  cudaFreeAsync(buf, st);
  cudaStreamSynchronize(st);
  return s;
}

}  // namespace

void amg_internal_free_fine(amg_coarse* h) {
  cudaFree(h->fU);
  if (h->fC != (void*)h->clover) cudaFree(h->fC);
  cudaFree(h->fwork);
  h->fU = h->fC = h->fwork = nullptr;
  h->fwork_bytes = 0;
}

extern "C" {

amg_status amg_setup_fine(amg_handle h, const void* d_U, void* stream) {
  if (!h || !d_U || !aligned16(d_U)) return AMG_ERR_INVALID_ARG;
  if (h->level != 1) return AMG_ERR_UNSUPPORTED;  // a level-2 handle has no fine lattice
  if (h->p.vec_prec != AMG_FP64 && h->p.vec_prec != AMG_FP32) return AMG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  amg_internal_free_fine(h);
  const long long nU = h->g.V * 36;
  if (fine_fp64(h)) {
    AMG_CUDA_TRY(cudaMalloc(&h->fU, nU * sizeof(double2)));
    AMG_CUDA_TRY(cudaMemcpyAsync(h->fU, d_U, nU * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    h->fC = h->clover;
  } else {
    AMG_CUDA_TRY(cudaMalloc(&h->fU, nU * sizeof(float2)));
    AMG_CUDA_TRY(cudaMalloc(&h->fC, h->g.V * kClPacked * sizeof(float2)));
    to_prec_kernel<float><<<4 * amg_sm_count(), 256, 0, st>>>((const double2*)d_U, (float2*)h->fU, nU);
    AMG_LAUNCH_CHECK();
    clover_pack_kernel<<<4 * amg_sm_count(), 256, 0, st>>>(h->clover, (float2*)h->fC, h->g.V);
    AMG_LAUNCH_CHECK();
    h->launches += 2;
  }
  return AMG_OK;
}

amg_status amg_dirac_apply(amg_handle h, const void* d_psi, void* d_out, int nrhs, void* stream) {
  AMG_TRY_INTERNAL(check_fine(h, d_psi, d_out, nrhs));
  if (d_psi == d_out) return AMG_ERR_INVALID_ARG;
  h->last_stream = (cudaStream_t)stream;
  return dirac_any(h, d_psi, nullptr, d_out, nrhs, (cudaStream_t)stream);
}

amg_status amg_sap(amg_handle h, const void* d_y, void* d_x, int nrhs, int n_cycles, int n_mr, void* stream) {
  AMG_TRY_INTERNAL(check_fine(h, d_y, d_x, nrhs));
  if (d_y == d_x || n_cycles < 0 || n_mr < 1) return AMG_ERR_INVALID_ARG;
  if (!sap_supported(h)) return AMG_ERR_UNSUPPORTED;
  h->last_stream = (cudaStream_t)stream;
  return sap_any(h, d_y, d_x, nrhs, n_cycles, n_mr, (cudaStream_t)stream);
}

amg_status amg_vcycle(amg_handle h, const amg_vcycle_params* vp, const void* d_y, void* d_x, int nrhs,
                      void* stream) {
  AMG_TRY_INTERNAL(check_fine(h, d_y, d_x, nrhs));
  AMG_TRY_INTERNAL(check_vp(vp));
  if (d_y == d_x) return AMG_ERR_INVALID_ARG;
  if (!sap_supported(h)) return AMG_ERR_UNSUPPORTED;
  h->last_stream = (cudaStream_t)stream;
  return vcycle_impl(h, vp, d_y, d_x, nrhs, (cudaStream_t)stream);
}

amg_status amg_adaptive_setup(amg_handle h, const amg_vcycle_params* vp, const void* d_U, void* d_tv, int n_setup,
                              void* stream) {
  if (!h || !d_U || !d_tv || !aligned16(d_U) || !aligned16(d_tv) || n_setup < 0) return AMG_ERR_INVALID_ARG;
  AMG_TRY_INTERNAL(check_vp(vp));
  if (h->next) return AMG_ERR_INVALID_ARG;  // an attached level 2 would keep D_cc of the old D_c
  if (!h->fU) return AMG_ERR_UNSUPPORTED;
  if (!sap_supported(h)) return AMG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  return fine_fp64(h) ? adaptive_impl<double>(h, vp, (const double2*)d_U, (double2*)d_tv, n_setup, st)
                      : adaptive_impl<float>(h, vp, (const double2*)d_U, (double2*)d_tv, n_setup, st);
}

amg_status amg_solve(amg_handle h, const amg_vcycle_params* vp, const void* d_f, void* d_u, int nrhs, double tol,
                     int restart, int max_applies, void* stream, double* info) {
  AMG_TRY_INTERNAL(check_fine(h, d_f, d_u, nrhs));
  AMG_TRY_INTERNAL(check_vp(vp));
  if (d_f == d_u || !(tol >= 0) || restart < 1 || restart > 64 || max_applies < 1) return AMG_ERR_INVALID_ARG;
  if (!sap_supported(h)) return AMG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  return fine_fp64(h) ? solve_impl<double>(h, vp, d_f, d_u, nrhs, tol, restart, max_applies, st, info)
                      : solve_impl<float>(h, vp, d_f, d_u, nrhs, tol, restart, max_applies, st, info);
}

}  // extern "C"
