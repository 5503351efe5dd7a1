// Internal declarations of libamg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include "../../include/amg.h"

#define AMG_MAX_NTV 64
#define AMG_NDIR 9

// Bits of the device error word.
#define AMG_EBIT_RANK 1u
#define AMG_EBIT_NONFINITE 2u
#define AMG_EBIT_TIMEOUT 4u
#define AMG_EBIT_INDEX 8u

// ---------------------------------------------------------------- geometry
struct Geom {
  int L[4], B[4], Lc[4];
  long long V, Vb, Vc;
  int ntv, nc, nagg;        // nc = 2 ntv, nagg = 6 Vb (dof per aggregate)
  const int* soff = nullptr;  // device: lattice offset of block-local site s from the block origin
};

__host__ __device__ inline long long site_index(const int* L, int x, int y, int z, int t) {
  return (((long long)t * L[2] + z) * L[1] + y) * L[0] + x;
}

// Fine site of local site s (lexicographic, x fastest) in block blk.
__host__ __device__ inline long long block_site(const Geom& g, long long blk, int s) {
  int X = (int)(blk % g.Lc[0]);
  long long r = blk / g.Lc[0];
  int Y = (int)(r % g.Lc[1]);
  r /= g.Lc[1];
  int Z = (int)(r % g.Lc[2]);
  int T = (int)(r / g.Lc[2]);
  int bx = s % g.B[0];
  int q = s / g.B[0];
  int by = q % g.B[1];
  q /= g.B[1];
  int bz = q % g.B[2];
  int bt = q / g.B[2];
  return site_index(g.L, X * g.B[0] + bx, Y * g.B[1] + by, Z * g.B[2] + bz, T * g.B[3] + bt);
}

// Fine site of the first site (local coordinates 0) of block blk.
__host__ __device__ inline long long block_origin(const Geom& g, long long blk) {
  const int X = (int)(blk % g.Lc[0]);
  long long r = blk / g.Lc[0];
  const int Y = (int)(r % g.Lc[1]);
  r /= g.Lc[1];
  const int Z = (int)(r % g.Lc[2]);
  const int T = (int)(r / g.Lc[2]);
  return site_index(g.L, X * g.B[0], Y * g.B[1], Z * g.B[2], T * g.B[3]);
}

// block_site through the precomputed offsets: origin + soff[s] (device code; g.soff set).
__device__ inline long long block_site_fast(const Geom& g, long long origin, int s) { return origin + __ldg(g.soff + s); }

// ---------------------------------------------------------------- complex helpers
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline void cfma(double2& acc, double2 a, double2 b) {  // acc += a b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__host__ __device__ inline void cfmac(double2& acc, double2 a, double2 b) {  // acc += conj(a) b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
__host__ __device__ inline void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__host__ __device__ inline void cfmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

// ---------------------------------------------------------------- handle
// Workspace of the coarse solve: one device buffer (Krylov basis, partial sums, scalars, flags),
// a mapped pinned word the device writes when a solve has converged, and a ring of events (one
// per Arnoldi step) after which the host reads it.
struct SolveWork {
  static constexpr int kRing = 16;
  void* buf = nullptr;
  size_t bytes = 0;
  int* hflag = nullptr;     // mapped pinned word: ticket of the last solve found converged
  int* hdone_dev = nullptr;  // its device address
  int ticket = 0;
  unsigned test_extra_arrivals = 0;  // test hook: arrivals the Arnoldi step's grid barrier waits for in vain
  cudaEvent_t ev[kRing] = {};
};

// Work buffer and launch shape of the fused batch (owned by the batch's first handle).
struct BatchWork {
  void* buf = nullptr;
  size_t bytes = 0;
  unsigned long long sig = 0;  // description of the batch whose job list is in buf
  int ns = 0, threads = 0, per_sm = 0;  // launch shape chosen by amg_batch_autotune (0: defaults)
  int test_extra_need = 0;     // test hook: jobs of phase 1 of lattice 0 that never arrive
};

struct amg_coarse {
  amg_params p;
  Geom g;
  double2* clover = nullptr;  // [V][2][6][6]
  double2* R64 = nullptr;     // [Nblock][2][ntv][6Vb], R_i^h row j = conj(q_j)
  void* Rq = nullptr;         // R in r_prec (aliases R64 for FP64)
  double2* Dc64 = nullptr;    // [Vc][9][nc][nc] canonical
  void* Dq = nullptr;         // D_c in link_prec, apply layout [Vc][9][nc col][nc row]
  float* Dscale = nullptr;    // [Vc][9] (FP16 scaled)
  void* Dtc = nullptr;        // BF16 tensor-core layout (when link_prec == BF16)
  void* Rtc = nullptr;        // BF16 tensor-core layout of R (when r_prec == BF16)
  void* tc_x = nullptr;       // BF16 planes of the coarse input of the tensor-core apply
  size_t tc_xbytes = 0;
  void* Dtf = nullptr;        // FP32 planes of D_c for the multi-RHS 3 x TF32 apply (link_prec FP32)
  void* tf_x = nullptr;       // FP32 rows of its coarse input
  size_t tf_xbytes = 0;
  int* nbr = nullptr;         // [Vc][9]
  double2* Dinv64 = nullptr;  // even/odd: inverses of the odd sites' self blocks [Vc/2][nc][nc] (row-major)
  void* Dinvq = nullptr;      // the same in link_prec, apply layout [Vc/2][nc col][nc row]
  int* eo_site = nullptr;     // [2][Vc/2]: site of half index h of parity p
  void* eo_tmp = nullptr;     // even/odd half vectors (solve workspace)
  size_t eo_tmp_bytes = 0;
  int* soff = nullptr;        // [Vb] site offsets inside a block (g.soff points here)
  unsigned int* err = nullptr;  // device error word
  float setup_ms[4] = {0, 0, 0, 0};
  cudaStream_t last_stream = 0;
  SolveWork sw;
  BatchWork bw;
  void* xc_tmp = nullptr;     // coarse scratch for amg_cgc
  void* yc_tmp = nullptr;
  size_t tmp_bytes = 0;
  unsigned long long launches = 0;  // kernels launched through this handle (host-side count)
  int grid_cap = 0;           // test hook: most CTAs of a grid-stride launch (0: occupancy x SMs)
  void* tc5_x = nullptr;      // tcgen05 apply (FP32 / FP16 storage, 4-16 columns): coarse rows,
  size_t tc5_xbytes = 0;
  float* tc5_xs = nullptr;    // their power-of-two scale per site,
  float* tc5_ds = nullptr;    // the power-of-two scale of every FP32 stencil block,
  void* tc5_d16 = nullptr;    // and the FP16 storage as planes with rotated pieces
  void* fU = nullptr;         // fine operator (amg_setup_fine): links [V][4][3][3] in vec_prec
  void* fC = nullptr;         // clover [V][2][6][6] in vec_prec (aliases clover for FP64)
  void* fwork = nullptr;      // outer FGMRES workspace (fine Krylov basis, Z vectors, sums)
  size_t fwork_bytes = 0;
  // Three levels (level2.cu).  A level-2 handle (level == 2) holds R2 in R64 ([Vc2][2][ntv2]
  // [Vb2 ntv1], row j = conj(q_j)), D_cc in Dc64 / Dq and its neighbour table; its geometry g has
  // L = the level-1 lattice, B = the level-2 blocks, V = Vc1 and nagg = Vb2 ntv1.
  int level = 1;
  amg_coarse* next = nullptr;  // level 1: the attached level-2 handle (its two-grid cycle replaces the coarse solve)
  amg_coarse* prev = nullptr;  // level 2: the level-1 handle it is attached to
  amg_level2_params l2p = {};  // level 1: the two-grid cycle's parameters
  void* l2work = nullptr;      // level 1: two level-1 and two level-2 vectors of the two-grid cycle
  size_t l2work_bytes = 0;
};

// Grid of a grid-stride launch over `items` work items with `resident` CTAs resident at once: the
// smaller of the two, lowered to the handle's test cap when one is set.
inline int capped_grid(const amg_coarse* h, long long items, long long resident) {
  long long g = items < resident ? items : resident;
  if (h->grid_cap > 0 && g > h->grid_cap) g = h->grid_cap;
  return (int)g;
}

// ---------------------------------------------------------------- shared host helpers
// Records the failing CUDA call of the calling thread (read back by amg_last_error()).
void amg_note_cuda_error(const char* file, int line, cudaError_t e);
// Records a printf-style message as the calling thread's last error.
void amg_note_error(const char* fmt, ...);

#define AMG_CUDA_TRY(call)                                \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      amg_note_cuda_error(__FILE__, __LINE__, e_);        \
      return e_ == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA; \
    }                                                     \
  } while (0)

#define AMG_LAUNCH_CHECK()                                \
  do {                                                    \
    cudaError_t e_ = cudaGetLastError();                  \
    if (e_ != cudaSuccess) {                              \
      amg_note_cuda_error(__FILE__, __LINE__, e_);        \
      return AMG_ERR_CUDA;                                \
    }                                                     \
  } while (0)

#define AMG_TRY_INTERNAL(call)          \
  do {                                  \
    amg_status s_ = (call);             \
    if (s_ != AMG_OK) return s_;        \
  } while (0)

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Streaming multiprocessors of the current device (queried once per device, api.cu); grids of
// the grid-stride kernels are multiples of it.
int amg_sm_count();

inline size_t vec_elem_bytes(amg_prec p) {
  return p == AMG_FP64 ? 16 : (p == AMG_FP32 ? 8 : 4);
}
inline size_t coarse_elem_bytes(const amg_coarse* h) { return h->p.vec_prec == AMG_FP64 ? 16 : 8; }

// Entry points of the translation units, used by the C ABI layer.
// Three levels: the coarse-grid correction of the fine level with the attached level-2 handle's
// two-grid cycle in place of the coarse solve (restriction, one two-grid cycle, prolongation).
amg_status amg_internal_cgc3(amg_coarse* h, const void* y, void* x, int nrhs, cudaStream_t s);
amg_status amg_internal_setup(amg_coarse* h, const double2* U, const double2* tv, cudaStream_t s);
// assembly partial sums ([Vc][5 jobs][2 slots][nc][nc], the layout combine_kernel reads) in pairs of floats
amg_status amg_internal_assemble_pair(const Geom& g, const double2* R, const double2* U, const double2* clov,
                                      double2* part, double m0, unsigned* err, cudaStream_t st);
// Gram-Schmidt per aggregate in pairs of floats (AMG_ERR_UNSUPPORTED above 1536 entries per aggregate)
amg_status amg_internal_gs_pair(const Geom& g, const double2* tv, double2* R, unsigned* err, cudaStream_t st);
amg_status amg_internal_restrict(amg_coarse* h, const void* y, void* yc, int nrhs, cudaStream_t s);
amg_status amg_internal_apply(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s);
amg_status amg_internal_prolong(amg_coarse* h, const void* xc, void* x, int nrhs, cudaStream_t s);
amg_status amg_internal_solve(amg_coarse* h, const void* b, void* x, int nrhs, double tol,
                              int restart, int max_applies, cudaStream_t s, double* info);
// The solve on a caller-provided workspace of amg_internal_solve_bytes() bytes; poll = false
// launches the whole budget without host events (kernels after convergence return at once).
amg_status amg_internal_solve_ws(amg_coarse* h, const void* b, void* x, int nrhs, double tol, int restart,
                                 int max_applies, cudaStream_t s, double* info, void* ws, bool poll);
size_t amg_internal_solve_bytes(const amg_coarse* h, int nrhs, int m);
amg_status amg_internal_batch(amg_coarse* const* hs, int n, const void* const* y, void* const* x,
                              const int* nrhs, cudaStream_t s);
amg_status amg_internal_export_stored(amg_coarse* h, double2* out);
amg_status amg_internal_tc_prepare(amg_coarse* h, cudaStream_t s);
void amg_internal_free_tc(amg_coarse* h);
void amg_internal_free_fine(amg_coarse* h);
// Rebuilds R and D_c (and every copy derived from them) from new test vectors on an existing
// handle: the setup of Alg. 5 again (api.cu); even/odd data are dropped (amg_setup_evenodd again).
amg_status amg_internal_rebuild(amg_coarse* h, const double2* U, const double2* tv, cudaStream_t s);
// Coarse application for the solver: CTAs return at once while *skip != 0; with xscale the input
// is xc * xscale[r] and that scaled input is also stored to vout (both may be null).
// Even/odd stencil piece (see eo_apply_kernel in stream.cu); parity of the output half.
amg_status amg_internal_eo_apply(amg_coarse* h, int parity, int d0, int d1, bool inv0, const void* s0, bool sc0,
                                 const void* s1, double c1, bool sc1, const void* vadd, double delta, void* y,
                                 void* vout, const double* xscale, const int* skip, int nrhs, cudaStream_t st,
                                 bool post_inv = false);
// y_e = S x_e with the Schur complement S = D_ee - D_eo D_oo^-1 D_oe (evenodd.cu); same extras as
// amg_internal_apply_ex, for the FGMRES driver.
amg_status amg_internal_schur_apply(amg_coarse* h, const void* xe, void* ye, int nrhs, cudaStream_t s,
                                    const int* skip, const double* xscale, void* vout);
typedef amg_status (*amg_apply_fn)(amg_coarse*, const void*, void*, int, cudaStream_t, const int*, const double*,
                                   void*);
// FGMRES on an operator over `rows` coarse rows (Vc nc for D_c, Vc nc / 2 for the Schur complement).
amg_status amg_internal_solve_op(amg_coarse* h, long long rows, amg_apply_fn op, const void* b, void* x, int nrhs,
                                 double tol, int restart, int max_applies, cudaStream_t s, double* info);
// FP32 D_c, nrhs = 4, 8, 12 or 16: tensor cores with split TF32 operands (tc.cu)
amg_status amg_internal_apply_tf32(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s,
                                   const int* skip, const double* xscale, void* vout);
// FP32 or FP16-scaled storage, 1 <= nrhs <= 16, nc % 8 == 0, nc <= 56: tcgen05 with FP16 split
// operands (tc5.cu); prepare allocates its storage at setup, free releases it.
bool amg_internal_tc5_supported(const amg_coarse* h);
amg_status amg_internal_tc5_prepare(amg_coarse* h, cudaStream_t s);
void amg_internal_free_tc5(amg_coarse* h);
amg_status amg_internal_apply_tc5(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s,
                                  const int* skip, const double* xscale, void* vout);
amg_status amg_internal_apply_ex(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s,
                                 const int* skip, const double* xscale, void* vout);
// Tensor-core (BF16) forms for nrhs = 4, 8, 12, 16.
amg_status amg_internal_apply_tc(amg_coarse* h, const void* xc, void* yc, int nrhs, cudaStream_t s,
                                 const int* skip, const double* xscale, void* vout);
amg_status amg_internal_restrict_tc(amg_coarse* h, const void* y, void* yc, int nrhs, cudaStream_t s);
amg_status amg_internal_prolong_tc(amg_coarse* h, const void* xc, void* x, int nrhs, cudaStream_t s);
