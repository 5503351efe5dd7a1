// Device implementation of the seeded synthetic-input generator (see synth/rng.py and
// synth/inputs.py for the definition, which this file implements independently):
// SplitMix64 output function over (seed, stream, counter), Box-Muller normals, complex
// Gaussians, and SU(3) links U = exp(i eps H), H = sum_a h_a lambda_a / 2.
// It computes nothing of the multigrid method.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace {

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t stream_base(uint64_t seed, uint64_t stream) {
  return mix64(mix64(seed) ^ (stream * 0xD1B54A32D192ED03ull));
}
__device__ inline double uniform(uint64_t base, uint64_t counter) {
  const uint64_t d = mix64(base + (counter + 1) * 0x9E3779B97F4A7C15ull);
  return ((double)(d >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}
// complex Gaussian m: Box-Muller pair from uniforms 2m, 2m+1
__device__ inline double2 cgauss(uint64_t base, uint64_t m) {
  const double u1 = uniform(base, 2 * m), u2 = uniform(base, 2 * m + 1);
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincos(2.0 * M_PI * u2, &s, &c);
  return make_double2(r * c, r * s);
}
__device__ inline double normal(uint64_t base, uint64_t k) {
  const double2 z = cgauss(base, k >> 1);
  return (k & 1) ? z.y : z.x;
}

struct C3 {
  double2 e[9];
};
__device__ inline double2 cm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline C3 mul(const C3& a, const C3& b) {
  C3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0, 0);
      for (int k = 0; k < 3; ++k) {
        const double2 t = cm(a.e[i * 3 + k], b.e[k * 3 + j]);
        s.x += t.x;
        s.y += t.y;
      }
      c.e[i * 3 + j] = s;
    }
  return c;
}

// U = exp(i eps H) by scaling and squaring with a degree-18 Taylor polynomial (Horner form).
__global__ void links_kernel(double2* out, long long V, double eps, uint64_t base) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= V * 4) return;
  double h[8];
  for (int a = 0; a < 8; ++a) h[a] = normal(base, (uint64_t)idx * 8 + a);
  const double r3 = 1.0 / sqrt(3.0);
  // H = sum h_a lambda_a / 2
  double2 H[9];
  H[0] = make_double2(0.5 * (h[2] + h[7] * r3), 0);
  H[4] = make_double2(0.5 * (-h[2] + h[7] * r3), 0);
  H[8] = make_double2(-h[7] * r3, 0);
  H[1] = make_double2(0.5 * h[0], -0.5 * h[1]);
  H[3] = make_double2(0.5 * h[0], 0.5 * h[1]);
  H[2] = make_double2(0.5 * h[3], -0.5 * h[4]);
  H[6] = make_double2(0.5 * h[3], 0.5 * h[4]);
  H[5] = make_double2(0.5 * h[5], -0.5 * h[6]);
  H[7] = make_double2(0.5 * h[5], 0.5 * h[6]);
  double nf = 0;
  for (int k = 0; k < 9; ++k) nf += H[k].x * H[k].x + H[k].y * H[k].y;
  nf = eps * sqrt(nf);
  int s = 0;
  while (nf > 0.5) {
    nf *= 0.5;
    ++s;
  }
  const double f = eps / (double)(1ll << s);
  C3 A;  // A = i f H
  for (int k = 0; k < 9; ++k) A.e[k] = make_double2(-f * H[k].y, f * H[k].x);
  C3 E;
  for (int k = 0; k < 9; ++k) E.e[k] = make_double2((k % 4 == 0) ? 1.0 : 0.0, 0);
  for (int n = 18; n >= 1; --n) {  // E = 1 + A/n E
    C3 t = mul(A, E);
    for (int k = 0; k < 9; ++k)
      E.e[k] = make_double2(((k % 4 == 0) ? 1.0 : 0.0) + t.e[k].x / n, t.e[k].y / n);
  }
  for (int q = 0; q < s; ++q) E = mul(E, E);
  double2* o = out + idx * 9;
  for (int k = 0; k < 9; ++k) o[k] = E.e[k];
}

// out[(n * ncols + j)] = cgauss(stream, index(n, j)); n = fine dof (site*12 + spin*3 + colour)
__global__ void tv_kernel(double2* out, long long ndof, int ntv, uint64_t base) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= ndof * ntv) return;
  const long long n = e / ntv;
  const int j = (int)(e % ntv);
  out[e] = cgauss(base, (uint64_t)n * 64 + j);
}

template <typename T>
__device__ inline T cast2(double2 v);
template <> __device__ inline double2 cast2<double2>(double2 v) { return v; }
template <> __device__ inline float2 cast2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }

template <typename T>
__global__ void rhs_kernel(T* out, long long ndof, int nrhs, uint64_t seed, uint64_t stream0) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= ndof * nrhs) return;
  const long long n = e / nrhs;
  const int r = (int)(e % nrhs);
  out[e] = cast2<T>(cgauss(stream_base(seed, stream0 + r), (uint64_t)n));
}

template <typename T>
__global__ void coarse_kernel(T* out, long long Vc, int ntv, int nrhs, uint64_t seed) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = Vc * 2 * ntv * nrhs;
  if (e >= total) return;
  const int r = (int)(e % nrhs);
  const long long q = e / nrhs;
  const int j = (int)(q % ntv);
  const int h = (int)((q / ntv) % 2);
  const long long i = q / (2 * ntv);
  out[e] = cast2<T>(cgauss(stream_base(seed, 1000 + r), (uint64_t)(i * 128 + h * 64 + j)));
}

inline unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" {

// Links [V][4][3][3] complex double.
int synth_links(void* d_out, long long V, double eps, unsigned long long seed, void* stream) {
  links_kernel<<<nblocks(V * 4, 128), 128, 0, (cudaStream_t)stream>>>((double2*)d_out, V, eps,
                                                                       stream_base(seed, 0));
  return (int)cudaGetLastError();
}

// Test vectors [V][4][3][ntv] complex double.
int synth_test_vectors(void* d_out, long long V, int ntv, unsigned long long seed, void* stream) {
  tv_kernel<<<nblocks(V * 12 * ntv, 256), 256, 0, (cudaStream_t)stream>>>((double2*)d_out, V * 12, ntv,
                                                                           stream_base(seed, 1));
  return (int)cudaGetLastError();
}

// Fine right-hand sides [V][4][3][nrhs]; prec 0 = complex double, 1 = complex float.
int synth_fine_rhs(void* d_out, long long V, int nrhs, unsigned long long seed, int prec, void* stream) {
  const long long n = V * 12 * nrhs;
  if (prec == 0)
    rhs_kernel<double2><<<nblocks(n, 256), 256, 0, (cudaStream_t)stream>>>((double2*)d_out, V * 12, nrhs, seed, 2);
  else
    rhs_kernel<float2><<<nblocks(n, 256), 256, 0, (cudaStream_t)stream>>>((float2*)d_out, V * 12, nrhs, seed, 2);
  return (int)cudaGetLastError();
}

// Coarse vectors [Vc][2][ntv][nrhs]; prec 0 = complex double, 1 = complex float.
int synth_coarse_vector(void* d_out, long long Vc, int ntv, int nrhs, unsigned long long seed, int prec,
                        void* stream) {
  const long long n = Vc * 2 * ntv * nrhs;
  if (prec == 0)
    coarse_kernel<double2><<<nblocks(n, 256), 256, 0, (cudaStream_t)stream>>>((double2*)d_out, Vc, ntv, nrhs, seed);
  else
    coarse_kernel<float2><<<nblocks(n, 256), 256, 0, (cudaStream_t)stream>>>((float2*)d_out, Vc, ntv, nrhs, seed);
  return (int)cudaGetLastError();
}

}  // extern "C"
