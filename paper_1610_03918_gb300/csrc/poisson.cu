// Field side of the step: charge density, the Poisson solve of Eq. 5 and
// E = -grad Phi (Sec. II).
//
// rho = sum_s q_s w_s 2^-20 acc_s + rho_ext + bottom surface charge; on the
// free (non-Dirichlet) nodes b = rho + sum of Dirichlet neighbour values.
// A = -Delta_h (5-point, unit spacing) on the free nodes, periodic where the
// box is.  rho and the potential are held as double-float pairs (hi + lo,
// about 48 bits; FP64 arithmetic runs at a small fraction of the FP32 rate
// on GB300).  The solve is an iterative refinement around an FP32 inner
// solve:
//
//   repeat:  r = rho - A phi        (double-float stencil over the whole
//                                    potential, Dirichlet values included:
//                                    the certificate)
//            stop if ||r|| <= rtol ||b||
//            solve A e = r          (FP32: the direct solve of fastpoisson.cu
//                                    where the geometry allows it, else PCG
//                                    with a symmetric V-cycle preconditioner,
//                                    inner products by FP32 tree sums, CG
//                                    coefficients in FP64)
//            phi += e               (double-float; the direct solve's
//                                    kernels add their parts of e in place)
//
// V-cycle: factor-2 coarsening with injected Dirichlet masks; Galerkin coarse
// operators A_c = R A P (9-point, built once on the host) with bilinear
// prolongation P and full-weighting restriction R = P^T / 4; red-black
// Gauss-Seidel on the 5-point fine level and four-colour Gauss-Seidel on the
// 9-point coarse levels, colours swept in reverse after the coarse
// correction, so the preconditioner is symmetric.  Levels with at most
// kSmallLevel nodes run inside one CTA with their vectors in shared memory.
// A doubly periodic box has no Dirichlet node: b loses its mean and the
// preconditioned residual is projected to zero mean.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>

#include "internal.cuh"

namespace picgb {
namespace {

constexpr int kThreads = 256;
#ifndef PICGB_SMALL_LEVEL
#define PICGB_SMALL_LEVEL 1024
#endif
constexpr int kSmallLevel = PICGB_SMALL_LEVEL;
#ifndef PICGB_COARSE_THREADS
#define PICGB_COARSE_THREADS 256
#endif
constexpr int kCoarseThreads = PICGB_COARSE_THREADS;
constexpr int kMaxOuter = 8;
constexpr int kCoarsestSweeps = 16;
#ifndef PICGB_DENSE_COARSEST
#define PICGB_DENSE_COARSEST 160
#endif
constexpr int kDenseCoarsest = PICGB_DENSE_COARSEST;   // coarsest levels with at most this many unknowns are solved exactly
constexpr size_t kCoarseSmemMax = 220 * 1024;   // dynamic shared memory granted to k_coarse
// A coarse-level stencil entry: the 3x3 Galerkin coefficients, then the
// reciprocal of the diagonal, padded to 48 bytes for 16-byte vector loads.
constexpr int kSt = 12;

// byte counts rounded up to 16: arrays staged into shared memory by 16-byte
// asynchronous copies are allocated with this padding
__host__ __device__ constexpr size_t pad16(size_t b) { return (b + 15) & ~size_t(15); }

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Cross-warp part of a block sum: lane 0 of each warp holds its warp's
// partials in v; thread 0 gets the block totals.
template <int NV>
__device__ void block_sum_warps(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][w] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0;
      for (int q = 0; q < nw; ++q) s += sh[k][q];
      v[k] = s;
    }
  }
  __syncthreads();
}

// Sum of NV doubles over the block; thread 0 gets the result.
template <int NV>
__device__ void block_sum(double (&v)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  block_sum_warps<NV>(v);
}

// Sums of squares for the norms, in FP32 without overflow or underflow:
// |x| in [2^-50, 2^50] is squared as it is, larger values after scaling by
// 2^-80 and smaller ones by 2^80, each class in its own accumulator (selects,
// no branch).  FP64 arithmetic is slow on GB300, so the grid sum runs in
// FP32 within each warp and in double-float pairs across warps and blocks;
// only the last step joins the classes in FP64.  The relative error of a
// norm is a few FP32 roundings.
struct SqSum {
  float mid, big, tiny;
};
__device__ __forceinline__ void sq_add(SqSum &a, float x) {
  const float ax = fabsf(x);
  const bool big = ax > 0x1p50f, tiny = ax < 0x1p-50f;
  const float y = x * (big ? 0x1p-80f : (tiny ? 0x1p80f : 1.f));
  const float y2 = y * y;
  a.mid += (big || tiny) ? 0.f : y2;
  a.big += big ? y2 : 0.f;
  a.tiny += tiny ? y2 : 0.f;
}

// Deterministic grid reduction: every block publishes its partials, the
// last block to arrive sums them in block order.  Returns true in the last
// block, where thread 0 holds the totals in v.  grid_sum_blocks starts from
// warp partials held by lane 0 of each warp.
template <int NV>
__device__ bool grid_sum_blocks(double (&v)[NV], double *part, unsigned int *ticket) {
  __shared__ bool last;
  block_sum_warps<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[blockIdx.x * NV + k] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  constexpr int kRound = NV >= 8 ? 1 : 8 / NV;   // partials per thread per round of loads
  double s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = 0;
  for (int b0 = threadIdx.x; b0 < (int)gridDim.x; b0 += kRound * blockDim.x) {
    double x[kRound][NV];
#pragma unroll
    for (int j = 0; j < kRound; ++j) {
      const int b = b0 + j * int(blockDim.x);
#pragma unroll
      for (int k = 0; k < NV; ++k) x[j][k] = b < (int)gridDim.x ? __ldcg(part + b * NV + k) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kRound; ++j)
#pragma unroll
      for (int k = 0; k < NV; ++k) s[k] += x[j][k];
  }
  block_sum<NV>(s);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = s[k];
    *ticket = 0u;
  }
  return true;
}

template <int NV>
__device__ bool grid_sum(double (&v)[NV], double *part, unsigned int *ticket) {
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  return grid_sum_blocks<NV>(v, part, ticket);
}


// FP32 tree sums of the sq_add classes.  Each block reduces its NC class
// sums by shuffles within the warps and then over the warps (block_tree,
// result in thread 0); the last block to arrive adds the blocks' partials
// the same way, in a fixed order.  The summands are non-negative, so each
// level of a tree adds at most one FP32 rounding to the relative error.
template <int NC>
__device__ __forceinline__ void block_tree(float (&c)[NC]) {
  __shared__ float sh[NC][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NC; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c[q] += __shfl_down_sync(0xffffffffu, c[q], o);
  __syncthreads();   // sh may still be read by a previous call
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NC; ++q) sh[q][w] = c[q];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      c[q] = lane < nw ? sh[q][lane] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c[q] += __shfl_down_sync(0xffffffffu, c[q], o);
    }
  }
}

// Publishes the block's sums (part[block][NC]) and takes a ticket; true in
// the last block to arrive.
template <int NC>
__device__ bool publish_sums(float (&c)[NC], float *part, unsigned int *ticket) {
  __shared__ bool last;
  block_tree<NC>(c);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NC; ++q) part[blockIdx.x * NC + q] = c[q];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  return last;
}

// In the last block: the totals of nb blocks' published sums, in thread 0.
template <int NC>
__device__ void sum_published(const float *part, int nb, float (&c)[NC]) {
  __threadfence();
#pragma unroll
  for (int q = 0; q < NC; ++q) c[q] = 0.f;
  for (int b0 = threadIdx.x; b0 < nb; b0 += 2 * blockDim.x) {   // both loads of a round in flight
    const int b1 = b0 + blockDim.x;
    float x[2][NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      x[0][q] = __ldcg(part + b0 * NC + q);
      x[1][q] = b1 < nb ? __ldcg(part + b1 * NC + q) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) c[q] += x[0][q] + x[1][q];
  }
  block_tree<NC>(c);
}

// Deterministic grid sum of FP32 per-thread partials (inner products of
// the PCG): FP32 tree sums within each block and over the blocks' published
// sums (fixed order), converted to FP64 once by thread 0 of the last block,
// where it returns true.  The partials buffer takes NV floats per block.
template <int NV>
__device__ bool grid_sum_f(const float (&s)[NV], double (&v)[NV], double *part, unsigned int *ticket) {
  float c[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) c[k] = s[k];
  float *pf = reinterpret_cast<float *>(part);
  if (!publish_sums<NV>(c, pf, ticket)) return false;
  sum_published<NV>(pf, gridDim.x, c);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = double(c[k]);
    *ticket = 0u;
  }
  return true;
}

// a class triple (mid, big, tiny) of sq_add as a double
__device__ __forceinline__ double sq_join(const float *c) {
  if (c[1] == 0.f && c[2] == 0.f) return double(c[0]);
  return double(c[0]) + double(c[1]) * 0x1p160 + double(c[2]) * 0x1p-160;
}

// sqrt(num / den) for finite num >= 0 and normal den > 0, to FP32 accuracy,
// without the FP64 divide and square root (long instruction sequences on
// GB300's narrow FP64 unit): the exponents are split off by bit
// manipulation and the mantissa ratio is taken in FP32.  NaN in, NaN out.
__device__ double sqrt_ratio(double num, double den) {
  if (num != num || den != den) return num + den;
  if (num == 0.0) return 0.0;
  if (num > 1.7e308) return num;
  const long long bn = __double_as_longlong(num), bd = __double_as_longlong(den);
  int e = int((bn >> 52) & 0x7ff) - int((bd >> 52) & 0x7ff);
  const float mn = __int_as_float(0x3f800000 | int((bn >> 29) & 0x7fffff));
  const float md = __int_as_float(0x3f800000 | int((bd >> 29) & 0x7fffff));
  float r = mn / md;
  if (e & 1) {
    r *= 2.f;
    e -= 1;
  }
  return double(sqrtf(r)) * __longlong_as_double((long long)(e / 2 + 1023) << 52);
}

struct FineArgs {
  Geom g;
  const uint8_t *flags;
  const float *lift;         // norms only
  const float2 *gval;
  float2 *rho, *phi;         // double-float
  float2 *phi_prev;          // potential of the previous step (extrapolated warm start)
  unsigned long long *acc;
  const float2 *rho_ext;
  const unsigned long long *bottom;
  float2 qw[2];              // q_s w_s 2^-20 (double-float)
  float2 sw[2];              // q_s w_s / 2: the charge of a surface hit on each of its two nodes
  int surface;
  float *r32, *z, *p, *w, *q, *e;
  PoissonState *ps;
  double *part;
  float *partf;              // the residual kernel's FP32 block sums
  float *bbpart;             // ||b||^2 block sums of a first pass that does not check
  unsigned int *ticket;
  int singular;
  int bb_from_part;          // the second pass takes ||b||^2 from bbpart
  double rtol;
  int maxit;
  int32_t *step;
  int advance_step;
  int init_solve;            // the density kernel also opens the next solve (resets its counters)
  float2 *E;
  double *fe;
  uint32_t *status;
  int graph;                 // kernels run inside the step graph: drive its conditionals
  int direct;                // the inner solve is the direct one (no inner loop)
  cudaGraphConditionalHandle h_outer, h_if_outer, h_inner, h_if_inner;
};

#define GRID_STRIDE(n, N) \
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < (N); n += gridDim.x * blockDim.x)

// The vector kernels take kVB nodes per thread, n = base + k * blockDim.x,
// and issue all loads of such a batch before its first store, so a thread
// waits for memory once per batch rather than once per node.
constexpr int kVB = 4;
#define VEC_BATCHES(base, N)                                                         \
  for (int base = blockIdx.x * blockDim.x * kVB + threadIdx.x; base < (N);          \
       base += gridDim.x * blockDim.x * kVB)
#define VEC_NODES(k, n, base, N)    \
  _Pragma("unroll") for (int k = 0; k < kVB; ++k) \
    if (const int n = (base) + k * int(blockDim.x); n < (N))

// rho at node n (double-float) from the species' deposit sums a0, a1, the
// external charge rx and, on the bottom row, the surface charge
__device__ __forceinline__ float2 node_rho(const FineArgs &a, const Geom &g, int n, unsigned long long a0,
                                           unsigned long long a1, float2 rx) {
  // two's-complement sums: a node's total can be slightly negative (CIC
  // shares of -1 unit from the fixed-point rounding)
  float2 rho = pair_add(pair_mul(a.qw[0], pair_from_ll((long long)a0)),
                        pair_mul(a.qw[1], pair_from_ll((long long)a1)));
  rho = pair_add(rx, rho);
  if (a.surface && !g.px) {
    const int i = fdiv(n, g.dnyn), j = n - i * g.nyn;
    if (i == g.nx - 1) {
      // half of bottom face k's charge on nodes (nx-1, k) and (nx-1, k+1)
      // (a.sw holds q_s w_s / 2)
      int jm = j - 1;
      if (g.py && jm < 0) jm += g.ny;
      if (j < g.ny)
        rho = pair_add(rho, pair_add(pair_mul(a.sw[0], pair_from_ll((long long)a.bottom[j])),
                                     pair_mul(a.sw[1], pair_from_ll((long long)a.bottom[g.ny + j]))));
      if (jm >= 0 && jm < g.ny)
        rho = pair_add(rho, pair_add(pair_mul(a.sw[0], pair_from_ll((long long)a.bottom[jm])),
                                     pair_mul(a.sw[1], pair_from_ll((long long)a.bottom[g.ny + jm]))));
    }
  }
  return rho;
}

// What the density kernel does once per launch (block 0, thread 0).
__device__ __forceinline__ void rho_bookkeeping(const FineArgs &a) {
  if (a.advance_step) *a.step += 1;
  if (a.init_solve) {
    a.ps->total_iters = 0;
    a.ps->outer_iters = 0;
  }
}

// acc -> rho (double-float); clears acc.  A doubly periodic box also forms
// the mean of rho, which the solve removes.
template <bool SING>
__global__ void k_rho(FineArgs a) {
  pdl_enter();
  const Geom g = a.g;
  const int nn = g.nxn * g.nyn;
  float2 sum = make_float2(0.f, 0.f);   // doubly periodic box: sum of rho
  VEC_BATCHES(base, nn) {
    unsigned long long a0[kVB], a1[kVB];
    float2 rx[kVB];
    VEC_NODES(k, n, base, nn) {
      a0[k] = a.acc[n];
      a1[k] = a.acc[nn + n];
      rx[k] = a.rho_ext[n];
    }
    VEC_NODES(k, n, base, nn) {
      a.acc[n] = 0ull;
      a.acc[nn + n] = 0ull;
      const float2 rho = node_rho(a, g, n, a0[k], a1[k], rx[k]);
      a.rho[n] = rho;
      if (SING) sum = pair_add(sum, rho);   // every node is free
    }
  }
  if (SING) {
    double v[1] = {pair_join(sum)};
    if (grid_sum<1>(v, a.part, a.ticket) && threadIdx.x == 0) a.ps->bmean = v[0] / double(nn);
  } else if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ps->bmean = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rho_bookkeeping(a);
}

// phi <- Dirichlet values, zero on free nodes (cold start)
__global__ void k_phi_reset(FineArgs a) {
  pdl_enter();
  GRID_STRIDE(n, a.g.nxn * a.g.nyn) a.phi[n] = a.gval[n];
}

// the lift start: phi <- phi_L, the potential of the empty box, on the free
// nodes (the Dirichlet nodes keep their values, which the RF bias moves)
__global__ void k_guess_lift(float2 *phi, const float2 *phiL, const uint8_t *flags, int nn) {
  pdl_enter();
  GRID_STRIDE(n, nn) {
    if (flags[n] & kFree) phi[n] = phiL[n];
  }
}

// initial guess extrapolated in time: phi <- 2 phi^n - phi^{n-1} on free nodes
__global__ void k_extrapolate(FineArgs a) {
  pdl_enter();
  const int nn = a.g.nxn * a.g.nyn;
  VEC_BATCHES(base, nn) {
    float2 p[kVB], q[kVB];
    uint8_t fl[kVB];
    VEC_NODES(k, n, base, nn) {
      fl[k] = a.flags[n];
      p[k] = a.phi[n];
      q[k] = a.phi_prev[n];
    }
    VEC_NODES(k, n, base, nn) {
      if (fl[k] & kFree) {
        a.phi[n] = pair_sub(make_float2(2.f * p[k].x, 2.f * p[k].y), q[k]);
        a.phi_prev[n] = p[k];
      }
    }
  }
}

__device__ __forceinline__ void nbr_index(const Geom &g, int n, int &xm, int &xp, int &ym, int &yp) {
  const int i = fdiv(n, g.dnyn), j = n - i * g.nyn;
  const int im = g.px ? wrapi(i - 1, g.nxn) : max(i - 1, 0);
  const int ip = g.px ? wrapi(i + 1, g.nxn) : min(i + 1, g.nxn - 1);
  const int jm = g.py ? wrapi(j - 1, g.nyn) : max(j - 1, 0);
  const int jp = g.py ? wrapi(j + 1, g.nyn) : min(j + 1, g.nyn - 1);
  xm = im * g.nyn + j;
  xp = ip * g.nyn + j;
  ym = i * g.nyn + jm;
  yp = i * g.nyn + jp;
}

// The difference a - b of two double-float values rounded to FP32: the high
// parts by TwoSum, the low parts and its error in FP32.
__device__ __forceinline__ float pair_diff(float2 a, float2 b) {
  const float2 t = two_sum(a.x, -b.x);
  return t.x + (t.y + (a.y - b.y));
}

// E = -grad phi at a node from its potential and its four neighbours' by the
// open-edge rule: a central difference where both edges along an axis border
// plasma, one-sided where one does, zero where neither does.
__device__ __forceinline__ float2 node_field(uint8_t fk, const float2 (&ph)[5]) {
  const bool xm = fk & kOpenXm, xp = fk & kOpenXp, ym = fk & kOpenYm, yp = fk & kOpenYp;
  const float2 x0 = xm ? ph[1] : ph[0], x1 = xp ? ph[2] : ph[0];
  const float2 y0 = ym ? ph[3] : ph[0], y1 = yp ? ph[4] : ph[0];
  const float ex = (xm || xp) ? -pair_diff(x1, x0) * ((xm && xp) ? 0.5f : 1.f) : 0.f;
  const float ey = (ym || yp) ? -pair_diff(y1, y0) * ((ym && yp) ? 0.5f : 1.f) : 0.f;
  return make_float2(ex, ey);
}

// r = rho - A phi at a free node = rho + phi_xm + phi_xp + phi_ym + phi_yp -
// 4 phi, rounded to FP32: the high parts are added by TwoSum, exactly, and
// the low parts with TwoSum's error terms in FP32, which leaves an error of
// a few units of 2^-46 |phi|.
__device__ __forceinline__ float resid_node(float2 rho, const float2 (&ph)[5]) {
  float2 s = two_sum(ph[1].x, ph[2].x);
  float2 t = two_sum(ph[3].x, ph[4].x);
  float lo = s.y + t.y;
  s = two_sum(s.x, t.x);
  lo += s.y;
  s = two_sum(s.x, -4.f * ph[0].x);
  lo += s.y;
  s = two_sum(s.x, rho.x);
  lo += s.y;
  lo += ((ph[1].y + ph[2].y) + (ph[3].y + ph[4].y)) - 4.f * ph[0].y + rho.y;
  return s.x + lo;
}

// Outer residual r = rho - A phi (the certificate; A applied to the whole
// potential, so the Dirichlet neighbour values enter through phi) from the
// double-float potential, and the set-up of the inner solve of A e = r.
// ||b||^2 (b = rho + lift on the free nodes) is formed on the first pass of
// a solve.  A checking pass (CHECK) also writes the field E of the potential
// it checks and its energy, so the pass that accepts the potential leaves
// the step's field, and decides whether the solve goes on.  A first pass
// known not to be the last (the direct solve's, which always corrects once)
// skips all that and leaves only its ||b||^2 block sums for the next pass.
template <bool CHECK, bool SING, bool FROM_ACC = false>
__global__ void k_resid(FineArgs a) {
  static_assert(!FROM_ACC || (!CHECK && !SING), "rho is formed only by a first pass without a check");
  pdl_enter();
  const Geom g = a.g;
  const int nn = g.nxn * g.nyn;
  // FROM_ACC: this kernel is the density kernel too, and so the solve's first pass
  const bool first = FROM_ACC || a.ps->outer_iters == 0;
  if (FROM_ACC && blockIdx.x == 0 && threadIdx.x == 0) {
    a.ps->bmean = 0.0;
    rho_bookkeeping(a);
  }
  const bool bb_here = first;
  float2 bm = make_float2(0.f, 0.f);
  if (SING) bm = pair_split(a.ps->bmean);
  SqSum q3[3] = {};
  VEC_BATCHES(base, nn) {
    float2 rh[kVB], ph[kVB][5];
    float lf[kVB];
    uint8_t fl[kVB];
    unsigned long long a0[FROM_ACC ? kVB : 1], a1[FROM_ACC ? kVB : 1];
    VEC_NODES(k, n, base, nn) {
      int xm, xp, ym, yp;
      nbr_index(g, n, xm, xp, ym, yp);
      fl[k] = a.flags[n];
      if (FROM_ACC) {
        a0[k] = a.acc[n];
        a1[k] = a.acc[nn + n];
        rh[k] = a.rho_ext[n];
      } else {
        rh[k] = a.rho[n];
      }
      lf[k] = bb_here ? a.lift[n] : 0.f;
      ph[k][0] = a.phi[n];
      ph[k][1] = a.phi[xm];
      ph[k][2] = a.phi[xp];
      ph[k][3] = a.phi[ym];
      ph[k][4] = a.phi[yp];
    }
    VEC_NODES(k, n, base, nn) {
      if (FROM_ACC) {
        a.acc[n] = 0ull;
        a.acc[nn + n] = 0ull;
        rh[k] = node_rho(a, g, n, a0[k], a1[k], rh[k]);
        a.rho[n] = rh[k];
      }
      float r32 = 0.f;
      if (fl[k] & kFree) {
        const float2 rho = SING ? pair_sub(rh[k], bm) : rh[k];
        r32 = resid_node(rho, ph[k]);
        if (CHECK) sq_add(q3[0], r32);
        if (bb_here) sq_add(q3[1], rho.x + (rho.y + lf[k]));
      }
      a.r32[n] = r32;
      if (CHECK) {
        const float2 E = node_field(fl[k], ph[k]);
        a.E[n] = E;
        sq_add(q3[2], E.x);
        sq_add(q3[2], E.y);
      }
      if (!a.direct) {             // the direct inner solve writes all of e and uses no p, q
        a.e[n] = 0.f;
        a.p[n] = 0.f;
        a.q[n] = 0.f;
      }
    }
  }
  if (!CHECK) {
    float cb[3] = {q3[1].mid, q3[1].big, q3[1].tiny};
    block_tree<3>(cb);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) a.bbpart[blockIdx.x * 3 + k] = cb[k];
    }
    return;
  }
  float c[9] = {q3[0].mid, q3[0].big, q3[0].tiny, q3[1].mid, q3[1].big, q3[1].tiny,
                q3[2].mid, q3[2].big, q3[2].tiny};
  if (!publish_sums<9>(c, a.partf, a.ticket)) return;
  sum_published<9>(a.partf, gridDim.x, c);
  PoissonState *ps = a.ps;
  const bool bb_parts = a.bb_from_part && ps->outer_iters == 1;
  float cb[3] = {0.f, 0.f, 0.f};
  if (bb_parts) sum_published<3>(a.bbpart, gridDim.x, cb);
  if (threadIdx.x == 0) {
    const double rr = sq_join(c);
    a.fe[0] = 0.5 * sq_join(c + 6);
    ps->rr64 = rr;
    if (first) ps->bb = sq_join(c + 3);
    if (bb_parts) ps->bb = sq_join(cb);
    const double bb = ps->bb;
    const float bbf = float(bb);
    if (c[1] == 0.f && c[2] == 0.f && bbf > 1e-30f && bbf < 1e30f)
      ps->rel = double(sqrtf(c[0] / bbf));   // both norms in FP32 range
    else
      ps->rel = sqrt_ratio(rr, bb > 0 ? bb : 1.0);
    if (first || bb_parts) ps->rel_first = ps->rel;
    const bool ok = ps->rel <= a.rtol || rr == 0.0;
    const bool give_up = !ok && ps->outer_iters >= kMaxOuter;
    if (give_up) atomicOr(a.status, PIC_ST_NOCONV);
    const bool go = !ok && !give_up;
    ps->outer_done = ok ? 1 : 0;
    ps->go = go ? 1 : 0;
    if (!go) {
      ps->n_solves += 1;
      ps->sum_outer += ps->outer_iters;
      ps->sum_total += ps->total_iters;
    }
    ps->inner_done = go ? 0 : 1;
    if (a.graph) {
      cudaGraphSetConditional(a.h_outer, go ? 1u : 0u);
      if (!a.direct) {
        cudaGraphSetConditional(a.h_if_outer, go ? 1u : 0u);
        cudaGraphSetConditional(a.h_inner, go ? 1u : 0u);
      }
    }
    ps->inner_iters = 0;
    ps->rr0 = rr;
    ps->rr = rr;
    // inner target: bring ||r|| to half the outer target (0.5 rtol / rel of
    // the initial residual), no tighter than FP32 allows
    const float t = 0.5f * float(a.rtol) / float(ps->rel);
    ps->tol_in = fminf(fmaxf(t, 3e-6f), 0.5f);
    ps->beta = 0.0;
    ps->rz = 0.0;
    *a.ticket = 0u;
  }
}

// The scalars after a preconditioner application z = M r, w = A z: zmean (a
// doubly periodic box projects z to zero mean, which leaves A z unchanged),
// gamma = <r, z - zmean> and delta = <z - zmean, w>.  v = {<r, z>, sum z,
// sum r, <z, w>, sum w}.
__device__ __forceinline__ void store_gamma_delta(PoissonState *ps, const double (&v)[5], int singular,
                                                  int nn) {
  const double zm = singular ? v[1] / double(nn) : 0.0;
  ps->zmean = zm;
  ps->rz = v[0] - zm * v[2];
  ps->delta = v[3] - zm * v[4];
  // the next CG step's coefficients (single-reduction form): once here
  // rather than in every thread of the update kernel
  const double gam = ps->rz;
  const bool first = ps->inner_iters == 0;
  const double beta = first ? 0.0 : gam / ps->rz_old;
  const double alpha = first ? gam / ps->delta : gam / (ps->delta - beta * gam / ps->alpha);
  ps->alpha_next = alpha;
  ps->beta_next = beta;
  ps->cg_f[0] = float(alpha);   // the update kernel's FP32 copies
  ps->cg_f[1] = float(beta);
  ps->cg_f[2] = float(zm);
}

// w = A z and the scalars of store_gamma_delta, after a V-cycle that ran
// entirely in one CTA (the tiled level-0 post-smoothing forms them otherwise)
__global__ void k_zw(FineArgs a) {
  pdl_enter();
  if (a.ps->inner_done) return;
  const Geom g = a.g;
  const int nn = g.nxn * g.nyn;
  float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  VEC_BATCHES(base, nn) {
    float z[kVB][5], r[kVB];
    uint8_t fl[kVB];
    VEC_NODES(k, n, base, nn) {
      int xm, xp, ym, yp;
      nbr_index(g, n, xm, xp, ym, yp);
      fl[k] = a.flags[n];
      r[k] = a.r32[n];
      z[k][0] = a.z[n];
      z[k][1] = a.z[xm];
      z[k][2] = a.z[xp];
      z[k][3] = a.z[ym];
      z[k][4] = a.z[yp];
    }
    VEC_NODES(k, n, base, nn) {
      // z is zero on the Dirichlet nodes, so the plain 5-point sum is A z
      const float w = (fl[k] & kFree) ? 4.f * z[k][0] - z[k][1] - z[k][2] - z[k][3] - z[k][4] : 0.f;
      a.w[n] = w;
      s[0] = fmaf(r[k], z[k][0], s[0]);
      s[1] += z[k][0];
      s[2] += r[k];
      s[3] = fmaf(z[k][0], w, s[3]);
      s[4] += w;
    }
  }
  double v[5];
  if (grid_sum_f<5>(s, v, a.part, a.ticket) && threadIdx.x == 0) store_gamma_delta(a.ps, v, a.singular, nn);
}

// One step of the preconditioned conjugate gradient in its single-reduction
// form (Chronopoulos and Gear): from gamma = <r, z>, delta = <z, A z> and the
// previous gamma and alpha,
//   beta = gamma / gamma_old,  alpha = gamma / (delta - beta gamma / alpha_old)
// (beta = 0, alpha = gamma / delta on the first step), then
//   p = (z - zmean) + beta p,  q = w + beta q (= A p),  e += alpha p,  r -= alpha q
// and rr = <r, r> for the convergence test.  The inner products of a step are
// all formed by the preconditioner's last kernel, so a step has one grid-wide
// reduction point besides this kernel's.
__global__ void k_cg(FineArgs a) {
  pdl_enter();
  PoissonState *ps = a.ps;
  if (ps->inner_done) return;
  const int nn = a.g.nxn * a.g.nyn;
  const float fa = ps->cg_f[0], fb = ps->cg_f[1], zm = ps->cg_f[2];
  float rr = 0.f;
  VEC_BATCHES(base, nn) {
    float z[kVB], w[kVB], p[kVB], q[kVB], e[kVB], r[kVB];
    VEC_NODES(k, n, base, nn) {
      z[k] = a.z[n];
      w[k] = a.w[n];
      p[k] = a.p[n];
      q[k] = a.q[n];
      e[k] = a.e[n];
      r[k] = a.r32[n];
    }
    VEC_NODES(k, n, base, nn) {
      const float pn = (z[k] - zm) + fb * p[k];
      const float qn = w[k] + fb * q[k];
      a.p[n] = pn;
      a.q[n] = qn;
      a.e[n] = e[k] + fa * pn;
      const float rn = r[k] - fa * qn;
      a.r32[n] = rn;
      rr = fmaf(rn, rn, rr);
    }
  }
  const float rs[1] = {rr};
  double v[1];
  if (grid_sum_f<1>(rs, v, a.part, a.ticket) && threadIdx.x == 0) {
    ps->rz_old = ps->rz;
    ps->alpha = ps->alpha_next;
    ps->beta = ps->beta_next;
    ps->rr = v[0];
    ps->inner_iters += 1;
    ps->total_iters += 1;
    const double tol = ps->tol_in;
    // ||r|| <= tol ||r_0||, compared as squares (no square roots)
    const bool done = v[0] <= tol * tol * ps->rr0 || ps->inner_iters >= a.maxit || !(v[0] == v[0]);
    if (done) ps->inner_done = 1;
    if (a.graph) {
      cudaGraphSetConditional(a.h_inner, done ? 0u : 1u);
      cudaGraphSetConditional(a.h_if_inner, done ? 0u : 1u);
    }
  }
}

__global__ void k_correct(FineArgs a) {
  pdl_enter();
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ps->outer_iters += 1;
  const int nn = a.g.nxn * a.g.nyn;
  VEC_BATCHES(base, nn) {
    float2 p[kVB];
    float e[kVB];
    uint8_t fl[kVB];
    VEC_NODES(k, n, base, nn) {
      fl[k] = a.flags[n];
      p[k] = a.phi[n];
      e[k] = a.e[n];
    }
    VEC_NODES(k, n, base, nn) {
      if (fl[k] & kFree) a.phi[n] = pair_add_f(p[k], e[k]);
    }
  }
}

__global__ void k_outer_init(PoissonState *ps) {
  pdl_enter();
  ps->total_iters = 0;
  ps->outer_iters = 0;
}

// E = -grad phi and the field energy 1/2 sum |E|^2 of the current potential
// (the residual kernel forms them too; this kernel serves the paths that
// change the potential without a solve)
__global__ void k_field(FineArgs a) {
  pdl_enter();
  const Geom g = a.g;
  const int nn = g.nxn * g.nyn;
  SqSum q1 = {};
  VEC_BATCHES(base, nn) {
    float2 ph[kVB][5];
    uint8_t fl[kVB];
    VEC_NODES(k, n, base, nn) {
      // neighbour indices clamped to the box; the edge flags say which count
      int xm, xp, ym, yp;
      nbr_index(g, n, xm, xp, ym, yp);
      fl[k] = a.flags[n];
      ph[k][0] = a.phi[n];
      ph[k][1] = a.phi[xm];
      ph[k][2] = a.phi[xp];
      ph[k][3] = a.phi[ym];
      ph[k][4] = a.phi[yp];
    }
    VEC_NODES(k, n, base, nn) {
      const float2 E = node_field(fl[k], ph[k]);
      a.E[n] = E;
      sq_add(q1, E.x);
      sq_add(q1, E.y);
    }
  }
  float c[3] = {q1.mid, q1.big, q1.tiny};
  if (!publish_sums<3>(c, a.partf, a.ticket)) return;
  sum_published<3>(a.partf, gridDim.x, c);
  if (threadIdx.x == 0) {
    a.fe[0] = 0.5 * sq_join(c);
    *a.ticket = 0u;
  }
}

// --------------------------------------------------------------------------
// Multigrid V-cycle
// --------------------------------------------------------------------------
struct LevelDev {
  int nxn, nyn, px, py;
  const uint8_t *free;   // level 0: 1 = unknown
  const uint16_t *sid;   // levels >= 1: 0 = not an unknown, k = stencil k-1 of stab
  const float *stab;     // levels >= 1: unique Galerkin stencils [k][kSt] (3x3, 1/diag)
  float *u, *f;
  float *upre;           // levels above lc: u after the pre-smoothing
};

struct MGArgs {
  LevelDev L[16];
  int nlev, lc;
  int nst[16];           // stencils per level
  int ncoarse;           // unknowns of the coarsest level solved by its dense inverse (0: sweeps)
  const float *cinv;     // [ncoarse][ncoarse]
  const int *cidx;       // node index of each coarsest unknown
  PoissonState *ps;
  float *w0;             // level 0: w = A z, formed by the post-smoothing
  double *part;          // its grid reduction of the PCG inner products
  unsigned int *ticket;
  int singular;
};

__device__ __forceinline__ int nb_idx(const LevelDev &L, int i, int j, int di, int dj) {
  const int a = L.px ? wrapi(i + di, L.nxn) : i + di;
  const int b = L.py ? wrapi(j + dj, L.nyn) : j + dj;
  return a * L.nyn + b;
}

template <bool FINE>
__device__ __forceinline__ bool is_free(const LevelDev &L, int n) {
  return FINE ? L.free[n] != 0 : L.sid[n] != 0;
}

// Off-diagonal part of (A u)(i, j) and the diagonal on level l: the 5-point
// unit Laplacian on the fine level, the node's Galerkin stencil on coarser
// ones.  Only called on free nodes, which are interior in a bounded direction.
template <bool FINE>
__device__ __forceinline__ float apply_off(const LevelDev &L, int i, int j, int n, float &diag,
                                           float &rdiag) {
  if (FINE) {
    diag = 4.f;
    rdiag = 0.25f;
    return -(L.u[nb_idx(L, i, j, -1, 0)] + L.u[nb_idx(L, i, j, 1, 0)] +
             L.u[nb_idx(L, i, j, 0, -1)] + L.u[nb_idx(L, i, j, 0, 1)]);
  } else {
    const float4 *s4 = reinterpret_cast<const float4 *>(L.stab + kSt * (int(L.sid[n]) - 1));
    const float4 a = s4[0], b = s4[1], c = s4[2];
    const float s[10] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y};
    diag = s[4];
    rdiag = s[9];
    float acc = 0.f;
#pragma unroll
    for (int di = -1; di <= 1; ++di)
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj) {
        if (di == 0 && dj == 0) continue;
        acc = fmaf(s[(di + 1) * 3 + (dj + 1)], L.u[nb_idx(L, i, j, di, dj)], acc);
      }
    return acc;
  }
}

// Gauss-Seidel update of one node of the current colour
template <bool FINE>
__device__ __forceinline__ void gs_node(const LevelDev &L, int i, int j) {
  const int n = i * L.nyn + j;
  if (!is_free<FINE>(L, n)) return;
  float d, rd;
  const float off = apply_off<FINE>(L, i, j, n, d, rd);
  L.u[n] = (L.f[n] - off) * rd;
}

// First half sweep from u = 0: the first colour gets f / diag, the rest 0.
template <bool FINE>
__device__ __forceinline__ void gs_zero_node(const LevelDev &L, int i, int j) {
  const int n = i * L.nyn + j;
  const bool first = FINE ? (((i + j) & 1) == 0) : (((i | j) & 1) == 0);
  float v = 0.f;
  if (first && is_free<FINE>(L, n))
    v = L.f[n] * (FINE ? 0.25f : L.stab[kSt * (int(L.sid[n]) - 1) + 9]);
  L.u[n] = v;
}

template <bool FINE>
__device__ __forceinline__ float resid_node(const LevelDev &L, int i, int j) {
  const int n = i * L.nyn + j;
  if (!is_free<FINE>(L, n)) return 0.f;
  float d, rd;
  const float off = apply_off<FINE>(L, i, j, n, d, rd);
  return L.f[n] - (d * L.u[n] + off);
}

// Full weighting of the fine residual onto coarse node (I, J) (0 where the
// coarse node is not an unknown).  It follows a forward sweep whose last
// colour has no neighbour of its own colour, so the residual there is zero up
// to rounding and is not evaluated: the black nodes, (a + b) odd, on the
// red-black level and the corners, a and b odd, on the four-colour levels.
// Five of the nine fine residuals remain.
template <bool FINE>
__device__ __forceinline__ float restrict_value(const LevelDev &F, const LevelDev &C, int I, int J) {
  if (!is_free<false>(C, I * C.nyn + J)) return 0.f;
  float s = 0.f;
#pragma unroll
  for (int a = -1; a <= 1; ++a) {
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      if (FINE ? ((a + b) & 1) != 0 : (a != 0 && b != 0)) continue;
      const int i = F.px ? wrapi(2 * I + a, F.nxn) : 2 * I + a;
      const int j = F.py ? wrapi(2 * J + b, F.nyn) : 2 * J + b;
      const float w = (a == 0 ? 2.f : 1.f) * (b == 0 ? 2.f : 1.f);
      s = fmaf(w, resid_node<FINE>(F, i, j), s);
    }
  }
  return s * (1.f / 16.f);
}

// bilinear prolongation of the coarse correction, added on free fine nodes
template <bool FINE>
__device__ __forceinline__ void prolong_node(const LevelDev &F, const LevelDev &C, int i, int j) {
  const int n = i * F.nyn + j;
  if (!is_free<FINE>(F, n)) return;
  const int I0 = i >> 1, J0 = j >> 1;
  const int I1 = (i & 1) ? (C.px ? wrapi(I0 + 1, C.nxn) : I0 + 1) : I0;
  const int J1 = (j & 1) ? (C.py ? wrapi(J0 + 1, C.nyn) : J0 + 1) : J0;
  const float v = 0.25f * (C.u[I0 * C.nyn + J0] + C.u[I1 * C.nyn + J0] + C.u[I0 * C.nyn + J1] +
                           C.u[I1 * C.nyn + J1]);
  F.u[n] += v;
}

// colour c of a level: fine level red/black (c in {0,1}, (i+j)&1 == c);
// coarse levels four colours (c in {0..3}, (i&1, j&1) == (c>>1, c&1)).
template <bool FINE>
__device__ __forceinline__ int colour_count(const LevelDev &L) {
  return FINE ? L.nxn * ((L.nyn + 1) >> 1) : ((L.nxn + 1) >> 1) * ((L.nyn + 1) >> 1);
}

// ---- the levels from lc down, inside one CTA, everything in shared memory ----
// The level descriptors are passed by value so their fields stay in registers.
//
// t / d for 0 <= t, d < 2^15 from the rounded reciprocal rd = 1/d: the
// rounded product differs from (t + 0.5) / d by less than 2^-23 (t + 0.5) / d,
// below that value's distance 0.5 / d to the nearest integer, so the
// truncation is exact (levels here hold at most 16384 nodes).
__device__ __forceinline__ int div_small(int t, float rd) {
  return int(__fmul_rn(__fadd_rn(float(t), 0.5f), rd));
}

template <bool FINE>
__device__ void cta_sweep(const LevelDev L, int c) {
  const int cnt = colour_count<FINE>(L);
  const int hy = (L.nyn + 1) >> 1;
  const float rhy = __frcp_rn(float(hy));
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const int ti = div_small(t, rhy);
    const int i = FINE ? ti : 2 * ti + (c >> 1);
    const int j = 2 * (t - ti * hy) + (FINE ? ((i + c) & 1) : (c & 1));
    if (i < L.nxn && j < L.nyn) gs_node<FINE>(L, i, j);
  }
  __syncthreads();
}

template <bool FINE>
__device__ void cta_zero(const LevelDev L) {
  const int nn = L.nxn * L.nyn;
  const float r = __frcp_rn(float(L.nyn));
  for (int n = threadIdx.x; n < nn; n += blockDim.x) {
    const int i = div_small(n, r);
    gs_zero_node<FINE>(L, i, n - i * L.nyn);
  }
  __syncthreads();
}

// forward sweep from colour c0, or a reverse sweep over all colours
template <bool FINE>
__device__ void cta_forward(const LevelDev L, int c0) {
  for (int c = c0; c < (FINE ? 2 : 4); ++c) cta_sweep<FINE>(L, c);
}

template <bool FINE>
__device__ void cta_backward(const LevelDev L) {
  for (int c = (FINE ? 1 : 3); c >= 0; --c) cta_sweep<FINE>(L, c);
}

// Restriction to level C; with `start` also the first half sweep of C from
// zero (colour 0 gets f / diag, the rest 0), which needs only the node's own f.
template <bool FINE>
__device__ void cta_restrict(const LevelDev F, const LevelDev C, bool start) {
  const int nn = C.nxn * C.nyn;
  const float r = __frcp_rn(float(C.nyn));
  for (int n = threadIdx.x; n < nn; n += blockDim.x) {
    const int I = div_small(n, r), J = n - I * C.nyn;
    const float v = restrict_value<FINE>(F, C, I, J);
    C.f[n] = v;
    if (start) {
      const int sid = C.sid[n];
      C.u[n] = (((I | J) & 1) == 0 && sid) ? v * C.stab[kSt * (sid - 1) + 9] : 0.f;
    }
  }
  __syncthreads();
}

template <bool FINE>
__device__ void cta_prolong(const LevelDev F, const LevelDev C) {
  const int nn = F.nxn * F.nyn;
  const float r = __frcp_rn(float(F.nyn));
  for (int n = threadIdx.x; n < nn; n += blockDim.x) {
    const int i = div_small(n, r);
    prolong_node<FINE>(F, C, i, n - i * F.nyn);
  }
  __syncthreads();
}

// ---- the levels above lc: each level's smoothing in two tiled kernels ----
//
// k_pre:  from u = 0, one forward sweep over the colours, then the full-
//         weighting restriction of the residual to level l+1.  A CTA owns a
//         TI x TJ block of coarse nodes; it repeats the sweep in shared memory
//         on every fine node those depend on (H = 2 nodes beyond the
//         restriction footprint on the red-black level, one per colour, 4, on
//         the four-colour levels), then writes the restricted residual of its
//         coarse nodes and the swept u of the fine nodes it owns to upre.
// k_post: u = upre + P u_{l+1} on the free nodes, then one reverse sweep.  A
//         CTA owns a PI x PJ block of fine nodes and repeats the work on the H
//         nodes around it.  It reads upre and writes u, so no CTA sees
//         another's writes.  On level 0 it also sums <r, z>, sum z and sum r
//         for the conjugate gradient.
// Colour c is swept at margin m from the edge of the shared region, with m
// growing by one per colour: a node at margin m reads neighbours at margin
// m - 1 or more, all of which the earlier colours have finished.
template <bool FINE> struct TileShape;
// H: halo of the pre-smoothing region, HP: of the post-smoothing region (one
// more on the red-black level, whose post-smoothing also forms w = A z)
template <> struct TileShape<true> {
  static constexpr int H = 2, HP = 3, TI = 8, TJ = 32, PI = 16, PJ = 64;
};
template <> struct TileShape<false> {
  static constexpr int H = 4, HP = 4, TI = 16, TJ = 16, PI = 16, PJ = 32;
};
constexpr int kTileThreads = 256;
constexpr int kTileStencils = 128;   // coarse stencil tables up to this size are staged in shared memory

template <bool FINE>
using NodeCode = typename std::conditional<FINE, uint8_t, uint16_t>::type;

template <bool FINE>
struct Tile {
  int gi0, gj0;          // level coordinates of region node (0, 0)
  int rh, rw;
  float *u, *f;
  NodeCode<FINE> *code;  // free flag / stencil id + 1; 0: not an unknown or outside the box
  const float *stab;
};

template <bool FINE>
__device__ __forceinline__ int tile_colour(const Tile<FINE> &T, int ri, int rj) {
  const int gi = T.gi0 + ri, gj = T.gj0 + rj;
  return FINE ? ((gi + gj) & 1) : (((gi & 1) << 1) | (gj & 1));
}

// off-diagonal part of (A u) at region node t, the diagonal and its reciprocal
template <bool FINE>
__device__ __forceinline__ float tile_off(const Tile<FINE> &T, int t, float &d, float &rd) {
  const float *u = T.u;
  const int w = T.rw;
  if (FINE) {
    d = 4.f;
    rd = 0.25f;
    return -(u[t - w] + u[t + w] + u[t - 1] + u[t + 1]);
  } else {
    const float4 *s4 = reinterpret_cast<const float4 *>(T.stab + kSt * (int(T.code[t]) - 1));
    const float4 a = s4[0], b = s4[1], c = s4[2];   // shared or global (large tables)
    d = b.x;
    rd = c.y;
    float acc = a.x * u[t - w - 1];
    acc = fmaf(a.y, u[t - w], acc);
    acc = fmaf(a.z, u[t - w + 1], acc);
    acc = fmaf(a.w, u[t - 1], acc);
    acc = fmaf(b.y, u[t + 1], acc);
    acc = fmaf(b.z, u[t + w - 1], acc);
    acc = fmaf(b.w, u[t + w], acc);
    acc = fmaf(c.x, u[t + w + 1], acc);
    return acc;
  }
}

template <bool FINE>
__device__ __forceinline__ float tile_resid(const Tile<FINE> &T, int t) {
  if (!T.code[t]) return 0.f;
  float d, rd;
  const float off = tile_off<FINE>(T, t, d, rd);
  return T.f[t] - (d * T.u[t] + off);
}

// One colour of a sweep on the region nodes at margin M or more; the threads
// are mapped onto the nodes of that colour only.
template <bool FINE, int RH, int RW, int M>
__device__ void tile_sweep(const Tile<FINE> &T, int c) {
  constexpr int W = (RW - 2 * M + 1) / 2;               // colour nodes per row (at most)
  constexpr int NR = FINE ? RH - 2 * M : (RH - 2 * M + 1) / 2;
  const int oi = ((c >> 1) - T.gi0 - M) & 1;             // four-colour row offset
  const int oj = FINE ? 0 : ((c & 1) - T.gj0 - M) & 1;
  for (int t = threadIdx.x; t < NR * W; t += blockDim.x) {
    const int a = t / W, b = t - a * W;
    const int ri = FINE ? M + a : M + 2 * a + oi;
    const int rj = FINE ? M + 2 * b + ((c - T.gi0 - ri - T.gj0 - M) & 1) : M + 2 * b + oj;
    if (ri >= RH - M || rj >= RW - M) continue;
    const int n = ri * RW + rj;
    if (!T.code[n]) continue;
    float d, rd;
    const float off = tile_off<FINE>(T, n, d, rd);
    T.u[n] = (T.f[n] - off) * rd;
  }
  __syncthreads();
}

__device__ __forceinline__ int wrap_mod(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// Coarse nodes under a fine region: rows from gi0 >> 1 to ((gi0 + RH - 1) >> 1) + 1.
template <int RH, int RW> struct CoarseBlock {
  static constexpr int CH = RH / 2 + 2, CW = RW / 2 + 2;
};

// Fills the region from level F in two parts.  Before the wait for the
// preceding kernel, the parts that never change during a solve: each node's
// free flag / stencil id and the stencil table.  After it: PRE: u = 0 except
// the first colour, which gets f / diag (the first half of the sweep from
// zero); otherwise u = upre plus the bilinear prolongation of level C's u
// (staged in cblk), on the free nodes.  Each thread takes K region nodes and
// issues all their loads before using any.  Returns false when the inner
// solve is already done.
template <bool FINE, bool PRE, int RH, int RW>
__device__ bool tile_load(const MGArgs &a, const LevelDev &F, const LevelDev &C, int nst,
                          Tile<FINE> &T, float *tab, float *cblk) {
  constexpr int N = RH * RW, K = (N + kTileThreads - 1) / kTileThreads;
  using CB = CoarseBlock<RH, RW>;
  int g[K], code[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int t = threadIdx.x + k * kTileThreads;
    const int ri = t / RW, rj = t - ri * RW;
    int gi = T.gi0 + ri, gj = T.gj0 + rj;
    bool in = t < N;
    if (F.px) gi = wrap_mod(gi, F.nxn);
    else in = in && gi >= 0 && gi < F.nxn;
    if (F.py) gj = wrap_mod(gj, F.nyn);
    else in = in && gj >= 0 && gj < F.nyn;
    g[k] = in ? gi * F.nyn + gj : -1;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) code[k] = g[k] >= 0 ? (FINE ? int(F.free[g[k]]) : int(F.sid[g[k]])) : 0;
  if (!FINE && nst <= kTileStencils) {
    for (int q = threadIdx.x; q < nst * kSt; q += blockDim.x) tab[q] = F.stab[q];
    T.stab = tab;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int t = threadIdx.x + k * kTileThreads;
    if (t < N) T.code[t] = NodeCode<FINE>(code[k]);
  }
  __syncthreads();
  pdl_enter();
  if (a.ps->inner_done) return false;
  float f[K], up[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    f[k] = 0.f;
    up[k] = 0.f;
    if (g[k] >= 0) {
      f[k] = F.f[g[k]];
      if (!PRE) up[k] = F.upre[g[k]];
    }
  }
  const int ci0 = T.gi0 >> 1, cj0 = T.gj0 >> 1;   // floor division
  if (!PRE) {
    for (int q = threadIdx.x; q < CB::CH * CB::CW; q += blockDim.x) {
      const int ca = q / CB::CW;
      int I = ci0 + ca, J = cj0 + (q - ca * CB::CW);
      bool in = true;
      if (C.px) I = wrap_mod(I, C.nxn);
      else in = I >= 0 && I < C.nxn;
      if (C.py) J = wrap_mod(J, C.nyn);
      else in = in && J >= 0 && J < C.nyn;
      cblk[q] = in ? C.u[I * C.nyn + J] : 0.f;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int t = threadIdx.x + k * kTileThreads;
    if (t >= N) break;
    const int ri = t / RW, rj = t - ri * RW;
    float u = 0.f;
    if (code[k]) {
      if (PRE) {
        if (tile_colour<FINE>(T, ri, rj) == 0)
          u = f[k] * (FINE ? 0.25f : T.stab[kSt * (code[k] - 1) + 9]);
      } else {
        const int gi = T.gi0 + ri, gj = T.gj0 + rj;
        const int a0 = (gi >> 1) - ci0, b0 = (gj >> 1) - cj0;
        const int a1 = a0 + (gi & 1), b1 = b0 + (gj & 1);
        u = up[k] + 0.25f * (cblk[a0 * CB::CW + b0] + cblk[a1 * CB::CW + b0] +
                             cblk[a0 * CB::CW + b1] + cblk[a1 * CB::CW + b1]);
      }
    }
    T.f[t] = f[k];
    T.u[t] = u;
  }
  __syncthreads();
  return true;
}

template <bool FINE>
__global__ void __launch_bounds__(kTileThreads) k_pre(MGArgs a, int l) {
  using S = TileShape<FINE>;
  static_assert(S::TI * S::TJ == kTileThreads, "one coarse node per thread");
  constexpr int RH = 2 * S::TI + 1 + 2 * S::H, RW = 2 * S::TJ + 1 + 2 * S::H;
  __shared__ float su[RH * RW], sf[RH * RW];
  __shared__ NodeCode<FINE> sc[RH * RW];
  __shared__ __align__(16) float tab[FINE ? 4 : kTileStencils * kSt];
  const LevelDev F = a.L[l], C = a.L[l + 1];
  const int tcj = (C.nyn + S::TJ - 1) / S::TJ;
  const int I0 = (blockIdx.x / tcj) * S::TI, J0 = (blockIdx.x % tcj) * S::TJ;
  // this thread's coarse node and whether it is an unknown (static)
  const int I = I0 + int(threadIdx.x) / S::TJ, J = J0 + int(threadIdx.x) % S::TJ;
  const bool own = I < C.nxn && J < C.nyn;
  const bool cfree = own && C.sid[I * C.nyn + J] != 0;
  Tile<FINE> T{2 * I0 - 1 - S::H, 2 * J0 - 1 - S::H, RH, RW, su, sf, sc, F.stab};
  if (!tile_load<FINE, true, RH, RW>(a, F, C, a.nst[l], T, tab, nullptr)) return;
  tile_sweep<FINE, RH, RW, 1>(T, 1);
  if (!FINE) {
    tile_sweep<FINE, RH, RW, 2>(T, 2);
    tile_sweep<FINE, RH, RW, 3>(T, 3);
  }
  // Restriction.  The last colour has no neighbour of its own colour, so its
  // residual after the sweep is zero up to rounding and is skipped: the black
  // nodes, (a + b) odd, on the red-black level and the corners, a and b odd,
  // on the four-colour levels.  Five of the nine fine residuals remain.
  if (own) {
    float sum = 0.f;
    if (cfree) {
      const int t0 = (2 * (I - I0) + 1 + S::H) * RW + 2 * (J - J0) + 1 + S::H;
#pragma unroll
      for (int da = -1; da <= 1; ++da)
#pragma unroll
        for (int db = -1; db <= 1; ++db) {
          if (FINE ? ((da + db) & 1) != 0 : (da != 0 && db != 0)) continue;
          const float w = (da == 0 ? 2.f : 1.f) * (db == 0 ? 2.f : 1.f);
          sum = fmaf(w, tile_resid<FINE>(T, t0 + da * RW + db), sum);
        }
      sum *= 1.f / 16.f;
    }
    C.f[I * C.nyn + J] = sum;
  }
  // the swept u of the fine nodes this tile owns
  for (int k = threadIdx.x; k < 4 * S::TI * S::TJ; k += blockDim.x) {
    const int ri = k / (2 * S::TJ), rj = k % (2 * S::TJ);
    const int i = 2 * I0 + ri, j = 2 * J0 + rj;
    if (i < F.nxn && j < F.nyn) F.upre[i * F.nyn + j] = su[(ri + 1 + S::H) * RW + rj + 1 + S::H];
  }
}

template <bool FINE>
__global__ void __launch_bounds__(kTileThreads) k_post(MGArgs a, int l) {
  using S = TileShape<FINE>;
  constexpr int RH = S::PI + 2 * S::HP, RW = S::PJ + 2 * S::HP;
  __shared__ float su[RH * RW], sf[RH * RW];
  __shared__ NodeCode<FINE> sc[RH * RW];
  __shared__ __align__(16) float tab[FINE ? 4 : kTileStencils * kSt];
  __shared__ float cblk[CoarseBlock<RH, RW>::CH * CoarseBlock<RH, RW>::CW];
  const LevelDev F = a.L[l], C = a.L[l + 1];
  const int tpj = (F.nyn + S::PJ - 1) / S::PJ;
  const int P0 = (blockIdx.x / tpj) * S::PI, Q0 = (blockIdx.x % tpj) * S::PJ;
  Tile<FINE> T{P0 - S::HP, Q0 - S::HP, RH, RW, su, sf, sc, F.stab};
  if (!tile_load<FINE, false, RH, RW>(a, F, C, a.nst[l], T, tab, cblk)) return;
  if (FINE) {
    tile_sweep<FINE, RH, RW, 1>(T, 1);
    tile_sweep<FINE, RH, RW, 2>(T, 0);
  } else {
    tile_sweep<FINE, RH, RW, 1>(T, 3);
    tile_sweep<FINE, RH, RW, 2>(T, 2);
    tile_sweep<FINE, RH, RW, 3>(T, 1);
    tile_sweep<FINE, RH, RW, 4>(T, 0);
  }
  float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  for (int k = threadIdx.x; k < S::PI * S::PJ; k += blockDim.x) {
    const int ri = k / S::PJ, rj = k % S::PJ;
    const int i = P0 + ri, j = Q0 + rj;
    if (i >= F.nxn || j >= F.nyn) continue;
    const int t = (ri + S::HP) * RW + rj + S::HP;
    const float z = su[t];
    const int n = i * F.nyn + j;
    F.u[n] = z;
    if (FINE) {
      // w = A z (z is zero on the Dirichlet nodes and outside the box)
      const float w = sc[t] ? 4.f * z - (su[t - RW] + su[t + RW] + su[t - 1] + su[t + 1]) : 0.f;
      a.w0[n] = w;
      const float r = sf[t];
      s[0] = fmaf(r, z, s[0]);
      s[1] += z;
      s[2] += r;
      s[3] = fmaf(z, w, s[3]);
      s[4] += w;
    }
  }
  if (!FINE) return;
  // level 0: u is the preconditioned residual z; the PCG scalars of the next step
  double v[5];
  if (grid_sum_f<5>(s, v, a.part, a.ticket) && threadIdx.x == 0)
    store_gamma_delta(a.ps, v, a.singular, F.nxn * F.nyn);
}

int pre_tiles(const MGLevel &C, bool fine) {
  const int ti = fine ? TileShape<true>::TI : TileShape<false>::TI;
  const int tj = fine ? TileShape<true>::TJ : TileShape<false>::TJ;
  return ((C.nxn + ti - 1) / ti) * ((C.nyn + tj - 1) / tj);
}

int post_tiles(const MGLevel &F, bool fine) {
  const int pi = fine ? TileShape<true>::PI : TileShape<false>::PI;
  const int pj = fine ? TileShape<true>::PJ : TileShape<false>::PJ;
  return ((F.nxn + pi - 1) / pi) * ((F.nyn + pj - 1) / pj);
}

// Asynchronous global -> shared copy of `bytes` (a multiple of 16, both
// addresses 16-byte aligned) in 16-byte pieces spread over the block; all of
// a block's copies are in flight together and cta_copy_wait ends them.
__device__ __forceinline__ void cta_copy_async(void *dst, const void *src, size_t bytes) {
  const unsigned d = unsigned(__cvta_generic_to_shared(dst));
  const char *g = static_cast<const char *>(src);
  for (size_t k = size_t(threadIdx.x) * 16; k < bytes; k += size_t(blockDim.x) * 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + unsigned(k)), "l"(g + k)
                 : "memory");
}

__device__ __forceinline__ void cta_copy_wait() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ T *carve(unsigned char *&p, size_t count) {
  T *r = reinterpret_cast<T *>(p);
  p += (count * sizeof(T) + 15) & ~size_t(15);
  return r;
}

// Shared-memory bytes of k_coarse (the same carving as the kernel).
size_t coarse_smem_bytes(const MGArgs &a) {
  auto seg = [](size_t b) { return (b + 15) & ~size_t(15); };
  size_t t = 0;
  for (int l = a.lc; l < a.nlev; ++l) {
    const size_t nn = size_t(a.L[l].nxn) * a.L[l].nyn;
    t += 2 * seg(nn * 4);
    t += l == 0 ? seg(nn) : seg(nn * 2) + seg(size_t(a.nst[l]) * kSt * 4);
  }
  t += seg(size_t(a.ncoarse) * a.ncoarse * 4) + seg(size_t(a.ncoarse) * 4);
  return t;
}

__global__ void __launch_bounds__(kCoarseThreads) k_coarse(MGArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  // level descriptors pointing into shared memory: one copy for the block
  __shared__ LevelDev S[16];
  const int lc = a.lc, last = a.nlev - 1;
  const int nc = a.ncoarse;
  // stage the level tables and the coarsest inverse (they do not change
  // during a solve, so before the wait for the preceding kernel), then the
  // first level's f
  unsigned char *p = smem;
  for (int l = lc; l <= last; ++l) {
    LevelDev L = a.L[l];
    const size_t nn = size_t(L.nxn) * L.nyn;
    L.u = carve<float>(p, nn);
    L.f = carve<float>(p, nn);
    if (l == 0) {
      uint8_t *fr = carve<uint8_t>(p, nn);
      cta_copy_async(fr, a.L[0].free, pad16(nn));
      L.free = fr;
    } else {
      uint16_t *sid = carve<uint16_t>(p, nn);
      float *tab = carve<float>(p, size_t(a.nst[l]) * kSt);
      cta_copy_async(sid, a.L[l].sid, pad16(nn * 2));
      cta_copy_async(tab, a.L[l].stab, size_t(a.nst[l]) * kSt * 4);
      L.sid = sid;
      L.stab = tab;
    }
    if (threadIdx.x == 0) S[l] = L;
  }
  __syncthreads();
  float *cinv = carve<float>(p, size_t(nc) * nc);
  int *cidx = carve<int>(p, nc);
  if (nc > 0) {
    cta_copy_async(cinv, a.cinv, pad16(size_t(nc) * nc * 4));
    cta_copy_async(cidx, a.cidx, pad16(size_t(nc) * 4));
    // the dense solve writes the unknowns only
    const int nn = S[last].nxn * S[last].nyn;
    for (int n = threadIdx.x; n < nn; n += blockDim.x) S[last].u[n] = 0.f;
  }
  pdl_enter();
  if (a.ps->inner_done) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }
  {
    const LevelDev &L = S[lc];
    cta_copy_async(L.f, a.L[lc].f, pad16(size_t(L.nxn) * L.nyn * 4));
  }
  cta_copy_wait();
  if (lc == 0) cta_zero<true>(S[lc]);
  else cta_zero<false>(S[lc]);
  for (int l = lc; l < last; ++l) {
    const bool start = !(l + 1 == last && nc > 0);
    if (l == 0) {
      cta_forward<true>(S[l], 1);
      cta_restrict<true>(S[l], S[l + 1], start);
    } else {
      cta_forward<false>(S[l], 1);
      cta_restrict<false>(S[l], S[l + 1], start);
    }
  }
  if (nc > 0) {
    // coarsest level: exact solve by the precomputed (pseudo-)inverse, a warp per row
    const LevelDev &L = S[last];
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < nc; r += nw) {
      float acc = 0.f;
      for (int k = lane; k < nc; k += 32) acc = fmaf(cinv[r * nc + k], L.f[cidx[k]], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) L.u[cidx[r]] = acc;
    }
    __syncthreads();
  } else if (last == 0) {
    cta_forward<true>(S[last], 1);
    for (int s = 1; s < kCoarsestSweeps; ++s) cta_forward<true>(S[last], 0);
    for (int s = 0; s < kCoarsestSweeps; ++s) cta_backward<true>(S[last]);
  } else {
    cta_forward<false>(S[last], 1);
    for (int s = 1; s < kCoarsestSweeps; ++s) cta_forward<false>(S[last], 0);
    for (int s = 0; s < kCoarsestSweeps; ++s) cta_backward<false>(S[last]);
  }
  for (int l = last - 1; l >= lc; --l) {
    if (l == 0) {
      cta_prolong<true>(S[l], S[l + 1]);
      cta_backward<true>(S[l]);
    } else {
      cta_prolong<false>(S[l], S[l + 1]);
      cta_backward<false>(S[l]);
    }
  }
  const int nn = S[lc].nxn * S[lc].nyn;
  for (int n = threadIdx.x; n < nn; n += blockDim.x) a.L[lc].u[n] = S[lc].u[n];
}

// --------------------------------------------------------------------------
// the residual kernel for the box: with or without the mean of rho removed
template <bool CHECK>
void (*resid_kernel(const pic_ctx *c))(FineArgs) {
  return c->singular ? k_resid<CHECK, true> : k_resid<CHECK, false>;
}

FineArgs fine_args(pic_ctx *c) {
  FineArgs a;
  a.g = c->g;
  a.flags = c->d_nodeflags;
  a.lift = c->d_lift;
  a.gval = c->d_g;
  a.rho = c->d_rho;
  a.phi = c->d_phi;
  a.phi_prev = c->d_phi_prev;
  a.acc = c->d_acc;
  a.rho_ext = c->d_rho_ext;
  // a decomposed run's rho takes the bottom counts summed over the ranks
  a.bottom = c->cfg.decomposed ? c->d_acc + 2 * size_t(c->g.nxn) * c->g.nyn : c->d_bottom;
  for (int s = 0; s < 2; ++s) {
    const double w = 1.0 / double(c->cfg.ppc[s]);
    a.qw[s] = pair_split(c->cfg.charge[s] * w * std::ldexp(1.0, -kFracBits));
    a.sw[s] = pair_split(0.5 * c->cfg.charge[s] * w);
  }
  a.surface = c->cfg.surface_charge;
  a.r32 = c->d_r32;
  a.z = c->d_z;
  a.p = c->d_p;
  a.w = c->d_w;
  a.q = c->d_q;
  a.e = c->d_e;
  a.ps = c->d_ps;
  a.part = c->red.part;
  a.partf = reinterpret_cast<float *>(c->red.part);
  a.bbpart = reinterpret_cast<float *>(c->red.part) + 16 * size_t(c->red.nblocks);
  a.ticket = c->red.ticket;
  a.singular = c->singular;
  a.bb_from_part = 0;
  a.rtol = c->cfg.poisson_rtol;
  a.maxit = c->cfg.poisson_maxit;
  a.step = c->d_step;
  a.advance_step = 0;
  a.init_solve = 0;
  a.E = c->d_E;
  a.fe = c->d_fe;
  a.status = c->d_status;
  a.graph = 0;
  a.direct = c->fp.enabled;
  a.h_outer = a.h_if_outer = a.h_inner = a.h_if_inner = 0;
  return a;
}

MGArgs mg_args(pic_ctx *c) {
  MGArgs a;
  a.nlev = c->nlev;
  a.lc = c->lc;
  for (int l = 0; l < c->nlev; ++l) {
    const MGLevel &m = c->lev[l];
    a.L[l].nxn = m.nxn;
    a.L[l].nyn = m.nyn;
    a.L[l].px = c->g.px;
    a.L[l].py = c->g.py;
    a.L[l].free = m.free;
    a.L[l].sid = m.sid;
    a.L[l].stab = m.stab;
    a.L[l].u = m.u;
    a.L[l].f = m.f;
    a.L[l].upre = m.upre;
    a.nst[l] = m.nst;
  }
  a.ncoarse = c->ncoarse;
  a.cinv = c->d_cinv;
  a.cidx = c->d_cidx;
  a.ps = c->d_ps;
  a.w0 = c->d_w;
  a.part = c->red.part;
  a.ticket = c->red.ticket;
  a.singular = c->singular;
  return a;
}

inline int blocks_for(int n) { return std::max(1, (n + kThreads - 1) / kThreads); }

// One V-cycle: the pre-smoothing and restriction of each level above lc, the
// levels from lc down in one CTA, then the prolongation and post-smoothing of
// each level back up.  With lc > 0 the last kernel also forms <r, z>.
void launch_vcycle(pic_ctx *c, const MGArgs &a) {
  for (int l = 0; l < c->lc; ++l) {
    const int nt = pre_tiles(c->lev[l + 1], l == 0);
    if (l == 0) launch(k_pre<true>, nt, kTileThreads, 0, c->stream, a, l);
    else launch(k_pre<false>, nt, kTileThreads, 0, c->stream, a, l);
  }
  launch(k_coarse, 1, kCoarseThreads, c->coarse_smem, c->stream, a);
  for (int l = c->lc - 1; l >= 0; --l) {
    const int nt = post_tiles(c->lev[l], l == 0);
    if (l == 0) launch(k_post<true>, nt, kTileThreads, 0, c->stream, a, l);
    else launch(k_post<false>, nt, kTileThreads, 0, c->stream, a, l);
  }
  c->launches += 2 * c->lc + 1;
}

// w = A z and the PCG scalars after a V-cycle that did not form them (every
// level in one CTA)
void launch_zw(pic_ctx *c, const FineArgs &f) {
  if (c->lc > 0) return;
  launch(k_zw, c->red.nblocks, kThreads, 0, c->stream, f);
  c->launches += 1;
}

// ---- host: Galerkin coarse operator A_c = R A_f P, R = P^T / 4 ----
// Fine stencils are 3x3 arrays per node (the 5-point unit Laplacian on
// level 0).  P is bilinear interpolation restricted to free nodes.
void galerkin(const Geom &g, int fnxn, int fnyn, const std::vector<uint8_t> &ffree,
              const std::vector<double> &fst, int cnxn, int cnyn, std::vector<uint8_t> &cfree,
              std::vector<double> &cst) {
  const bool px = g.px, py = g.py;
  auto wrapx = [&](int a, int n) { return px ? ((a % n) + n) % n : a; };
  auto wrapy = [&](int a, int n) { return py ? ((a % n) + n) % n : a; };
  auto half_floor = [](int a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); };
  cst.assign(size_t(cnxn) * cnyn * 9, 0.0);
  for (int I = 0; I < cnxn; ++I) {
    for (int J = 0; J < cnyn; ++J) {
      const size_t C = size_t(I) * cnyn + J;
      if (!cfree[C]) continue;
      double *out = &cst[C * 9];
      for (int a = -1; a <= 1; ++a) {
        for (int b = -1; b <= 1; ++b) {
          // fine node i = (2I + a, 2J + b) with P[i, C] = wa * wb
          const int fi_u = 2 * I + a, fj_u = 2 * J + b;
          const int fi = wrapx(fi_u, fnxn), fj = wrapy(fj_u, fnyn);
          if (fi < 0 || fi >= fnxn || fj < 0 || fj >= fnyn) continue;
          const size_t fidx = size_t(fi) * fnyn + fj;
          if (!ffree[fidx]) continue;
          const double wiC = (a == 0 ? 1.0 : 0.5) * (b == 0 ? 1.0 : 0.5) / 4.0;
          for (int di = -1; di <= 1; ++di) {
            for (int dj = -1; dj <= 1; ++dj) {
              const double coef = fst[fidx * 9 + (di + 1) * 3 + (dj + 1)];
              if (coef == 0.0) continue;
              // fine node j = i + (di, dj), unwrapped relative to 2C
              const int gi_u = fi_u + di, gj_u = fj_u + dj;
              const int gi = wrapx(gi_u, fnxn), gj = wrapy(gj_u, fnyn);
              if (gi < 0 || gi >= fnxn || gj < 0 || gj >= fnyn) continue;
              if (!ffree[size_t(gi) * fnyn + gj]) continue;
              // coarse nodes D with P[j, D] != 0 (unwrapped coordinates)
              const int dI0 = half_floor(gi_u), dJ0 = half_floor(gj_u);
              const bool oddi = (gi_u - 2 * dI0) != 0, oddj = (gj_u - 2 * dJ0) != 0;
              for (int sI = 0; sI <= (oddi ? 1 : 0); ++sI) {
                for (int sJ = 0; sJ <= (oddj ? 1 : 0); ++sJ) {
                  const int DI_u = dI0 + sI, DJ_u = dJ0 + sJ;
                  const double wjD = (oddi ? 0.5 : 1.0) * (oddj ? 0.5 : 1.0);
                  const int DI = wrapx(DI_u, cnxn), DJ = wrapy(DJ_u, cnyn);
                  if (DI < 0 || DI >= cnxn || DJ < 0 || DJ >= cnyn) continue;
                  if (!cfree[size_t(DI) * cnyn + DJ]) continue;
                  const int oI = DI_u - I, oJ = DJ_u - J;
                  if (oI < -1 || oI > 1 || oJ < -1 || oJ > 1) continue;
                  out[(oI + 1) * 3 + (oJ + 1)] += wiC * coef * wjD;
                }
              }
            }
          }
        }
      }
      if (!(out[4] > 0.0)) cfree[C] = 0;
    }
  }
}

}  // namespace

cudaError_t poisson_setup(pic_ctx *c) {
  const Geom &g = c->g;
  c->singular = 1;
  for (size_t n = 0; n < c->h_nodeflags.size(); ++n)
    if (!(c->h_nodeflags[n] & kFree)) c->singular = 0;
  // level hierarchy
  c->lev.clear();
  MGLevel L0;
  L0.nx = g.nx;
  L0.ny = g.ny;
  L0.nxn = g.nxn;
  L0.nyn = g.nyn;
  L0.h2 = 1.f;
  std::vector<std::vector<uint8_t>> masks;
  std::vector<std::vector<double>> sts;
  std::vector<uint8_t> m0(size_t(g.nxn) * g.nyn);
  for (size_t n = 0; n < m0.size(); ++n) m0[n] = (c->h_nodeflags[n] & kFree) ? 1 : 0;
  std::vector<double> s0(m0.size() * 9, 0.0);
  for (size_t n = 0; n < m0.size(); ++n) {
    if (!m0[n]) continue;
    double *s = &s0[n * 9];
    s[4] = 4.0;
    s[1] = s[3] = s[5] = s[7] = -1.0;
  }
  masks.push_back(m0);
  sts.push_back(s0);
  c->lev.push_back(L0);
  while (c->lev.size() < 16) {
    // a level with at most kDenseCoarsest unknowns is solved exactly: stop there
    size_t unknowns = 0;
    for (uint8_t v : masks.back()) unknowns += v;
    if (unknowns <= size_t(kDenseCoarsest)) break;
    const MGLevel &F = c->lev.back();
    const bool even = (F.nx % 2 == 0) && (F.ny % 2 == 0);
    if (!even) break;
    const int cnx = F.nx / 2, cny = F.ny / 2;
    if (cnx < 2 || cny < 2) break;
    if (g.px && (cnx % 2)) break;
    if (g.py && (cny % 2)) break;
    MGLevel C;
    C.nx = cnx;
    C.ny = cny;
    C.nxn = g.px ? cnx : cnx + 1;
    C.nyn = g.py ? cny : cny + 1;
    C.h2 = F.h2 * 4.f;
    std::vector<uint8_t> mc(size_t(C.nxn) * C.nyn);
    const std::vector<uint8_t> &mf = masks.back();
    for (int I = 0; I < C.nxn; ++I)
      for (int J = 0; J < C.nyn; ++J) mc[size_t(I) * C.nyn + J] = mf[size_t(2 * I) * F.nyn + 2 * J];
    std::vector<double> sc;
    galerkin(g, F.nxn, F.nyn, mf, sts.back(), C.nxn, C.nyn, mc, sc);
    masks.push_back(mc);
    sts.push_back(sc);
    c->lev.push_back(C);
  }
  c->nlev = int(c->lev.size());
  c->lc = c->nlev - 1;
  for (int l = 0; l < c->nlev; ++l)
    if (c->lev[l].nxn * c->lev[l].nyn <= kSmallLevel) {
      c->lc = l;
      break;
    }
  const size_t nn = size_t(g.nxn) * g.nyn;
  for (int l = 0; l < c->nlev; ++l) {
    MGLevel &m = c->lev[l];
    const size_t n = size_t(m.nxn) * m.nyn;
    m.free = nullptr;
    m.sid = nullptr;
    m.stab = nullptr;
    m.nst = 0;
    if (l == 0) {
      m.free = (uint8_t *)dev_alloc(c, pad16(n));
      if (!m.free) return cudaErrorMemoryAllocation;
      cudaMemcpy(m.free, masks[0].data(), n, cudaMemcpyHostToDevice);
      m.u = nullptr;
      m.f = nullptr;
      continue;
    }
    // unique stencils of the level and each node's entry (0 = not an unknown)
    std::map<std::array<float, 9>, int> table;
    std::vector<std::array<float, 9>> uniq;
    std::vector<uint16_t> sid(n, 0);
    for (size_t k = 0; k < n; ++k) {
      if (!masks[l][k]) continue;
      std::array<float, 9> st;
      for (int q = 0; q < 9; ++q) st[q] = float(sts[l][k * 9 + q]);
      auto it = table.find(st);
      int id;
      if (it == table.end()) {
        id = int(uniq.size());
        if (id >= 65535) return cudaErrorInvalidValue;
        table.emplace(st, id);
        uniq.push_back(st);
      } else {
        id = it->second;
      }
      sid[k] = uint16_t(id + 1);
    }
    m.nst = int(uniq.size());
    std::vector<float> tab(std::max<size_t>(uniq.size(), 1) * kSt, 0.f);
    for (size_t k = 0; k < uniq.size(); ++k) {
      for (int q = 0; q < 9; ++q) tab[k * kSt + q] = uniq[k][q];
      tab[k * kSt + 9] = 1.f / uniq[k][4];
    }
    m.sid = (uint16_t *)dev_alloc(c, pad16(n * 2));
    m.stab = (float *)dev_alloc(c, tab.size() * 4);
    m.u = (float *)dev_alloc(c, n * sizeof(float));
    m.f = (float *)dev_alloc(c, pad16(n * sizeof(float)));
    if (!m.u || !m.f || !m.sid || !m.stab) return cudaErrorMemoryAllocation;
    cudaMemcpy(m.sid, sid.data(), n * 2, cudaMemcpyHostToDevice);
    cudaMemcpy(m.stab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice);
    cudaMemsetAsync(m.u, 0, n * sizeof(float), c->stream);
    cudaMemsetAsync(m.f, 0, pad16(n * sizeof(float)), c->stream);
  }
  // coarsest level: dense (pseudo-)inverse when it is small
  {
    const int last = c->nlev - 1;
    const MGLevel &m = c->lev[last];
    const size_t n = size_t(m.nxn) * m.nyn;
    std::vector<int> idx;
    for (size_t k = 0; k < n; ++k)
      if (masks[last][k]) idx.push_back(int(k));
    const int nc = int(idx.size());
    c->ncoarse = 0;
    c->d_cinv = nullptr;
    c->d_cidx = nullptr;
    if (nc > 0 && nc <= kDenseCoarsest) {
      std::vector<int> pos(n, -1);
      for (int r = 0; r < nc; ++r) pos[idx[r]] = r;
      // dense operator over the unknowns (level 0: 5-point; else the Galerkin stencils)
      std::vector<double> A(size_t(nc) * nc, 0.0);
      for (int r = 0; r < nc; ++r) {
        const int I = idx[r] / m.nyn, J = idx[r] % m.nyn;
        for (int di = -1; di <= 1; ++di)
          for (int dj = -1; dj <= 1; ++dj) {
            const double coef = sts[last][size_t(idx[r]) * 9 + (di + 1) * 3 + (dj + 1)];
            if (coef == 0.0) continue;
            int a = I + di, b = J + dj;
            if (g.px) a = (a + m.nxn) % m.nxn;
            if (g.py) b = (b + m.nyn) % m.nyn;
            if (a < 0 || a >= m.nxn || b < 0 || b >= m.nyn) continue;
            const int q = pos[size_t(a) * m.nyn + b];
            if (q >= 0) A[size_t(r) * nc + q] += coef;
          }
      }
      // a doubly periodic box is singular (constants): invert A + 11^T/n, subtract 11^T/n
      if (c->singular)
        for (auto &v : A) v += 1.0 / nc;
      std::vector<double> inv(size_t(nc) * nc, 0.0);
      for (int r = 0; r < nc; ++r) inv[size_t(r) * nc + r] = 1.0;
      bool ok = true;
      for (int col = 0; col < nc && ok; ++col) {   // Gauss-Jordan with partial pivoting
        int piv = col;
        for (int r = col + 1; r < nc; ++r)
          if (std::fabs(A[size_t(r) * nc + col]) > std::fabs(A[size_t(piv) * nc + col])) piv = r;
        if (!(std::fabs(A[size_t(piv) * nc + col]) > 1e-300)) { ok = false; break; }
        if (piv != col)
          for (int k = 0; k < nc; ++k) {
            std::swap(A[size_t(piv) * nc + k], A[size_t(col) * nc + k]);
            std::swap(inv[size_t(piv) * nc + k], inv[size_t(col) * nc + k]);
          }
        const double d = A[size_t(col) * nc + col];
        for (int k = 0; k < nc; ++k) {
          A[size_t(col) * nc + k] /= d;
          inv[size_t(col) * nc + k] /= d;
        }
        for (int r = 0; r < nc; ++r) {
          if (r == col) continue;
          const double f = A[size_t(r) * nc + col];
          if (f == 0.0) continue;
          for (int k = 0; k < nc; ++k) {
            A[size_t(r) * nc + k] -= f * A[size_t(col) * nc + k];
            inv[size_t(r) * nc + k] -= f * inv[size_t(col) * nc + k];
          }
        }
      }
      if (ok) {
        if (c->singular)
          for (auto &v : inv) v -= 1.0 / nc;
        std::vector<float> invf(inv.begin(), inv.end());
        c->d_cinv = (float *)dev_alloc(c, pad16(invf.size() * 4));
        c->d_cidx = (int *)dev_alloc(c, pad16(idx.size() * 4));
        if (!c->d_cinv || !c->d_cidx) return cudaErrorMemoryAllocation;
        cudaMemcpy(c->d_cinv, invf.data(), invf.size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_cidx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice);
        c->ncoarse = nc;
      }
    }
  }
  c->coarse_smem = coarse_smem_bytes(mg_args(c));
  if (c->coarse_smem > kCoarseSmemMax) return cudaErrorInvalidValue;
  // the attribute belongs to the kernel, not to this context: always grant the
  // largest size any context may use, so contexts of different sizes coexist
  cudaError_t e = cudaFuncSetAttribute(k_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(kCoarseSmemMax));
  if (e != cudaSuccess) return e;
  float **vecs[] = {&c->d_r32, &c->d_z, &c->d_p, &c->d_w, &c->d_q, &c->d_e};
  for (float **v : vecs) {
    *v = (float *)dev_alloc(c, pad16(nn * sizeof(float)));
    if (!*v) return cudaErrorMemoryAllocation;
    cudaMemsetAsync(*v, 0, pad16(nn * sizeof(float)), c->stream);
  }
  c->lev[0].u = c->d_z;
  c->lev[0].f = c->d_r32;
  for (int l = 0; l < c->nlev; ++l) {
    MGLevel &m = c->lev[l];
    m.upre = nullptr;
    if (l >= c->lc) continue;
    m.upre = (float *)dev_alloc(c, size_t(m.nxn) * m.nyn * sizeof(float));
    if (!m.upre) return cudaErrorMemoryAllocation;
  }
  c->d_phi_prev = (float2 *)dev_alloc(c, nn * sizeof(float2));
  if (!c->d_phi_prev) return cudaErrorMemoryAllocation;
  // kVB nodes per thread in the vector kernels
  c->red.nblocks = blocks_for((int(nn) + kVB - 1) / kVB);
  // partials of the grid reductions: the vector kernels and the level-0 post-smoothing
  const int nparts = std::max(c->red.nblocks, c->lc > 0 ? post_tiles(c->lev[0], true) : 0);
  c->red.part = (double *)dev_alloc(c, size_t(nparts) * 16 * sizeof(double));
  c->red.ticket = (unsigned int *)dev_alloc(c, 64);
  c->d_ps = (PoissonState *)dev_alloc(c, sizeof(PoissonState));
  if (!c->red.part || !c->red.ticket || !c->d_ps) return cudaErrorMemoryAllocation;
  cudaMemsetAsync(c->red.ticket, 0, 64, c->stream);
  cudaMemsetAsync(c->d_ps, 0, sizeof(PoissonState), c->stream);
  e = cudaMallocHost((void **)&c->h_ps, sizeof(PoissonState));
  if (e != cudaSuccess) return e;
  cudaEventCreate(&c->ev0);
  cudaEventCreate(&c->ev1);
  e = fast_poisson_setup(c);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

bool rho_in_solve(const pic_ctx *c) {
  return c->fp.enabled && c->cfg.warm_start == 1 && !c->singular;
}

cudaError_t launch_rho(pic_ctx *c, int advance_step, int init_solve) {
  FineArgs a = fine_args(c);
  a.advance_step = advance_step;
  a.init_solve = init_solve;
  if (c->singular) launch(k_rho<true>, c->red.nblocks, kThreads, 0, c->stream, a);
  else launch(k_rho<false>, c->red.nblocks, kThreads, 0, c->stream, a);
  return cudaGetLastError();
}

cudaError_t launch_field(pic_ctx *c) {
  FineArgs a = fine_args(c);
  launch(k_field, c->red.nblocks, kThreads, 0, c->stream, a);
  return cudaGetLastError();
}

namespace {

struct RFArgs {
  const int32_t *dir;        // the electrode's Dirichlet nodes
  const float2 *g0;          // their static values
  int ndir;
  const int32_t *lnodes;     // free nodes next to them
  const float *cnt;          // their number of electrode neighbours
  const float *lift0;        // their static lift
  int nlift;
  float2 *phi, *gval;
  float *lift;
  const int32_t *step;
  int advance;
  double dt, amp, omega;
};

// RF bias (Sec. III-B): the electrode value at t = (step + advance) dt is the
// static value plus amp sin(omega t), written into the potential's and the
// Dirichlet data's electrode nodes; the lift of their free neighbours (used
// only for ||b||) follows.
__global__ void k_rf_bias(RFArgs a) {
  pdl_enter();
  const double t = double(*a.step + a.advance) * a.dt;
  const double v = a.amp * sin(a.omega * t);
  const float2 vp = pair_split(v);
  GRID_STRIDE(k, a.ndir) {
    const float2 gv = pair_add(a.g0[k], vp);
    a.phi[a.dir[k]] = gv;
    a.gval[a.dir[k]] = gv;
  }
  GRID_STRIDE(k, a.nlift) a.lift[a.lnodes[k]] = a.lift0[k] + float(v) * a.cnt[k];
}

}  // namespace

cudaError_t launch_rf_bias(pic_ctx *c, int advance) {
  if (c->cfg.phi_rf_amp == 0.0 || (c->n_rf_dir == 0 && c->n_rf_lift == 0)) return cudaSuccess;
  RFArgs a;
  a.dir = c->d_rf_dir;
  a.g0 = c->d_rf_g0;
  a.ndir = c->n_rf_dir;
  a.lnodes = c->d_rf_lift;
  a.cnt = c->d_rf_cnt;
  a.lift0 = c->d_rf_lift0;
  a.nlift = c->n_rf_lift;
  a.phi = c->d_phi;
  a.gval = c->d_g;
  a.lift = c->d_lift;
  a.step = c->d_step;
  a.advance = advance;
  a.dt = c->cfg.dt;
  a.amp = c->cfg.phi_rf_amp;
  a.omega = c->cfg.omega_rf;
  const int n = std::max(a.ndir, a.nlift);
  launch(k_rf_bias, std::max(1, std::min(64, (n + kThreads - 1) / kThreads)), kThreads, 0, c->stream, a);
  c->launches += 1;
  return cudaGetLastError();
}

pic_status poisson_solve(pic_ctx *c, bool zero_guess) {
  FineArgs a = fine_args(c);
  const MGArgs m = mg_args(c);
  const int nb = c->red.nblocks;
  cudaEventRecord(c->ev0, c->stream);
  if (zero_guess) {
    launch(k_phi_reset, nb, kThreads, 0, c->stream, a);
    c->launches += 1;
  } else if (c->cfg.warm_start == 2) {
    launch(k_extrapolate, nb, kThreads, 0, c->stream, a);
    c->launches += 1;
  } else if (c->cfg.warm_start == 3) {
    if (launch_learned_guess(c) != cudaSuccess) return PIC_ECUDA;
  } else if (c->cfg.warm_start == 4) {
    launch(k_guess_lift, nb, kThreads, 0, c->stream, c->d_phi, c->d_phiL, c->d_nodeflags,
           c->g.nxn * c->g.nyn);
    c->launches += 1;
  }
  launch(k_outer_init, 1, 1, 0, c->stream, c->d_ps);
  c->launches += 1;
  const int batch = 4;
  for (;;) {
    launch(resid_kernel<true>(c), nb, kThreads, 0, c->stream, a);
    c->launches += 1;
    cudaMemcpyAsync(c->h_ps, c->d_ps, sizeof(PoissonState), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
    if (!c->h_ps->go) break;
    if (c->fp.enabled) {   // the direct solve adds its correction to phi itself
      fast_poisson_launch(c, c->d_r32, c->d_phi, c->d_ps);
      continue;
    }
    launch_vcycle(c, m);
    launch_zw(c, a);
    for (int it = 0; it < c->cfg.poisson_maxit; it += batch) {
      for (int b = 0; b < batch; ++b) {
        launch(k_cg, nb, kThreads, 0, c->stream, a);
        launch_vcycle(c, m);
        launch_zw(c, a);
        c->launches += 1;
      }
      cudaMemcpyAsync(c->h_ps, c->d_ps, sizeof(PoissonState), cudaMemcpyDeviceToHost, c->stream);
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
      if (c->h_ps->inner_done) break;
    }
    launch(k_correct, nb, kThreads, 0, c->stream, a);
    c->launches += 1;
  }
  cudaEventRecord(c->ev1, c->stream);
  cudaMemcpyAsync(c->h_ps, c->d_ps, sizeof(PoissonState), cudaMemcpyDeviceToHost, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->last_ms = ms;
  c->last_outer = c->h_ps->outer_iters;
  // solves from the host loop count their own launches
  c->seen_solves = c->h_ps->n_solves;
  c->seen_outer = c->h_ps->sum_outer;
  c->seen_total = c->h_ps->sum_total;
  if (note(cudaGetLastError(), "Poisson solve") != cudaSuccess) return PIC_ECUDA;
  return c->h_ps->outer_done ? PIC_OK : PIC_ENOCONV;
}

// ---- the solve as nested conditional nodes of a CUDA graph ----
namespace {

cudaError_t cap_begin(cudaStream_t s, cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps) {
  return cudaStreamBeginCaptureToGraph(s, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                       deps.size(), cudaStreamCaptureModeThreadLocal);
}

cudaError_t cap_end(cudaStream_t s, std::vector<cudaGraphNode_t> &leaves) {
  cudaStreamCaptureStatus st;
  unsigned long long id;
  cudaGraph_t gg;
  const cudaGraphNode_t *d = nullptr;
  const cudaGraphEdgeData *ed = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, &id, &gg, &d, &ed, &nd);
  if (e != cudaSuccess) return e;
  leaves.assign(d, d + nd);
  cudaGraph_t out;
  return cudaStreamEndCapture(s, &out);
}

cudaError_t add_cond(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps,
                     cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                     cudaGraphNode_t *node, cudaGraph_t *body) {
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaError_t e = cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                   deps.size(), &p);
  if (e == cudaSuccess) *body = p.conditional.phGraph_out[0];
  return e;
}

}  // namespace

// Appends the solve to graph `top` after the nodes in `deps`; on return
// `deps` holds the solve's last node.  With the multigrid inner solve:
//   [phi reset] -> init -> WHILE(outer) { resid -> IF(go) { V-cycle ->
//     WHILE(inner) { cg -> IF(!done) { V-cycle } } -> correct } }
// where a V-cycle also forms w = A z and the inner products of the next step.
// With the direct inner solve, whose one pass nearly always suffices, the
// first pass runs unconditionally (a potential that already meets the
// tolerance takes one correction it does not need) and only further passes
// are conditional (the direct solve adds its correction to phi itself):
//   [phi reset] -> init -> resid -> solve -> resid -> WHILE(go) { solve -> resid }
cudaError_t poisson_capture(pic_ctx *c, cudaGraph_t top, std::vector<cudaGraphNode_t> &deps) {
  cudaStream_t s = c->stream;
  FineArgs a = fine_args(c);
  const MGArgs m = mg_args(c);
  const int nb = c->red.nblocks;
  const bool direct = c->fp.enabled;
  cudaGraphConditionalHandle h[4];
  const int nh = direct ? 1 : 4;
  for (int k = 0; k < nh; ++k) {
    cudaError_t e = cudaGraphConditionalHandleCreate(&h[k], top, (k == 0 && !direct) ? 1u : 0u,
                                                     cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return note(e, "cudaGraphConditionalHandleCreate");
  }
  a.graph = 1;
  a.h_outer = h[0];
  a.h_if_outer = direct ? 0 : h[1];
  a.h_inner = direct ? 0 : h[2];
  a.h_if_inner = direct ? 0 : h[3];
  cudaError_t e;
#define CK(x) do { if ((e = (x)) != cudaSuccess) { note(e, #x); return e; } } while (0)
  CK(cap_begin(s, top, deps));
  if (c->cfg.warm_start == 0) launch(k_phi_reset, nb, kThreads, 0, s, a);
  if (c->cfg.warm_start == 2) launch(k_extrapolate, nb, kThreads, 0, s, a);
  if (c->cfg.warm_start == 3) CK(launch_learned_guess(c));
  if (c->cfg.warm_start == 4)
    launch(k_guess_lift, nb, kThreads, 0, s, c->d_phi, c->d_phiL, c->d_nodeflags, c->g.nxn * c->g.nyn);
  // (with the previous step's potential as the guess the density kernel just
  // before opened the solve)
  if (c->cfg.warm_start != 1) launch(k_outer_init, 1, 1, 0, s, c->d_ps);
  if (direct) {
    // the first pass always corrects: it leaves ||b||^2 to the second
    if (rho_in_solve(c)) {   // and forms rho, opening the step's solve
      FineArgs r = a;
      r.advance_step = 1;
      r.init_solve = 1;
      launch(k_resid<false, false, true>, nb, kThreads, 0, s, r);
    } else {
      launch(resid_kernel<false>(c), nb, kThreads, 0, s, a);
    }
    fast_poisson_launch(c, c->d_r32, c->d_phi, c->d_ps);
    a.bb_from_part = 1;
    launch(resid_kernel<true>(c), nb, kThreads, 0, s, a);
  }
  CK(cap_end(s, deps));
  cudaGraphNode_t n_outer, n_if_outer, n_inner, n_if_inner;
  cudaGraph_t b_outer, b_if_outer, b_inner, b_if_inner;
  CK(add_cond(top, deps, h[0], cudaGraphCondTypeWhile, &n_outer, &b_outer));
  std::vector<cudaGraphNode_t> d;
  if (direct) {
    CK(cap_begin(s, b_outer, {}));
    fast_poisson_launch(c, c->d_r32, c->d_phi, c->d_ps);
    launch(resid_kernel<true>(c), nb, kThreads, 0, s, a);
    CK(cap_end(s, d));
    deps.assign(1, n_outer);
    return cudaGetLastError();
  }
  CK(cap_begin(s, b_outer, {}));
  launch(resid_kernel<true>(c), nb, kThreads, 0, s, a);
  CK(cap_end(s, d));
  CK(add_cond(b_outer, d, h[1], cudaGraphCondTypeIf, &n_if_outer, &b_if_outer));
  CK(cap_begin(s, b_if_outer, {}));
  launch_vcycle(c, m);
  launch_zw(c, a);
  CK(cap_end(s, d));
  CK(add_cond(b_if_outer, d, h[2], cudaGraphCondTypeWhile, &n_inner, &b_inner));
  CK(cap_begin(s, b_inner, {}));
  launch(k_cg, nb, kThreads, 0, s, a);
  CK(cap_end(s, d));
  CK(add_cond(b_inner, d, h[3], cudaGraphCondTypeIf, &n_if_inner, &b_if_inner));
  CK(cap_begin(s, b_if_inner, {}));
  launch_vcycle(c, m);
  launch_zw(c, a);
  CK(cap_end(s, d));
  d.assign(1, n_inner);
  CK(cap_begin(s, b_if_outer, d));
  launch(k_correct, nb, kThreads, 0, s, a);
  CK(cap_end(s, d));
#undef CK
  deps.assign(1, n_outer);
  return cudaGetLastError();
}

// Kernels that S solves with O outer passes and I inner iterations in all
// launched (graph mode; every outer pass takes at least one inner iteration).
int64_t poisson_kernel_count(pic_ctx *c, int64_t S, int64_t O, int64_t I) {
  // final resid, and unless the density kernel opens the solve: guess and init
  int64_t per_solve = 1 + (c->cfg.warm_start != 1 ? 2 : 0);
  if (c->cfg.warm_start == 3) per_solve += 2 + unet_forward_kernels();   // absmax, input, network
  if (c->fp.enabled)   // per pass: resid, direct solve (which corrects phi)
    return S * per_solve + O * (c->fp.kernels + 1);
  // a V-cycle with w = A z and the inner products: fused into its last kernel unless lc = 0
  const int64_t vc = 2 * c->lc + 1 + (c->lc == 0 ? 1 : 0);
  // per pass: resid, V-cycle, correct; per iteration: cg; per non-final iteration: V-cycle
  return S * per_solve + O * (vc + 2) + I + (I - O) * vc;
}


// ---- initial guesses for the learned warm start ----
namespace {

__global__ void k_absmax(const float2 *rho, int nn, unsigned int *out) {
  pdl_enter();
  float m = 0.f;
  GRID_STRIDE(n, nn) m = fmaxf(m, fabsf(rho[n].x));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));   // m >= 0: bit order = value order
}

// x[i][j] = (rho / s, 1 for a Dirichlet node); rows beyond the grid count as conductor
__global__ void k_learned_input(const float2 *rho, const uint8_t *flags, int nxn, int nyn, int hpad,
                                const unsigned int *smax, float *x) {
  pdl_enter();
  const float s = fmaxf(__uint_as_float(*smax), 1e-30f);
  GRID_STRIDE(n, hpad * nyn) {
    const int i = n / nyn;
    float r = 0.f, m = 1.f;
    if (i < nxn) {
      r = float(pair_join(rho[n]) / double(s));
      m = (flags[n] & kFree) ? 0.f : 1.f;
    }
    x[2 * n] = r;
    x[2 * n + 1] = m;
  }
}

__global__ void k_guess_learned(float2 *phi, const float2 *phiL, const uint8_t *flags, const float *y,
                                double scale, int nn) {
  pdl_enter();
  GRID_STRIDE(n, nn) {
    if (flags[n] & kFree) phi[n] = pair_split(pair_join(phiL[n]) + scale * double(y[n]));
  }
}

// the same with the scale s = max |rho| read on the device (the in-step guess)
__global__ void k_guess_learned_dev(float2 *phi, const float2 *phiL, const uint8_t *flags, const float *y,
                                    const unsigned int *smax, int nn) {
  pdl_enter();
  const double s = double(fmaxf(__uint_as_float(*smax), 1e-30f));
  GRID_STRIDE(n, nn) {
    if (flags[n] & kFree) phi[n] = pair_split(pair_join(phiL[n]) + s * double(y[n]));
  }
}

// training target of the warm-start network: (phi - phi_L) / s on the nodes,
// 0 on the padding rows
__global__ void k_learned_target(const float2 *phi, const float2 *phiL, int nn, int npad, double inv_s,
                                 float *t) {
  pdl_enter();
  GRID_STRIDE(n, npad) t[n] = n < nn ? float((pair_join(phi[n]) - pair_join(phiL[n])) * inv_s) : 0.f;
}

}  // namespace

// The potential of the empty box (Dirichlet values only), solved once to
// 1e-10 and kept.
pic_status ensure_vacuum_potential(pic_ctx *c) {
  if (c->d_phiL) return PIC_OK;
  const size_t nn = size_t(c->g.nxn) * c->g.nyn;
  c->d_phiL = (float2 *)dev_alloc(c, nn * 8);
  float2 *save_phi = (float2 *)dev_alloc(c, nn * 8);
  float2 *save_rho = (float2 *)dev_alloc(c, nn * 8);
  if (!c->d_phiL || !save_phi || !save_rho) return PIC_ENOMEM;
  cudaMemcpyAsync(save_phi, c->d_phi, nn * 8, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(save_rho, c->d_rho, nn * 8, cudaMemcpyDeviceToDevice, c->stream);
  PoissonState ps_save;
  cudaMemcpyAsync(&ps_save, c->d_ps, sizeof(ps_save), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  // no charge: b is the Dirichlet lift alone
  cudaMemsetAsync(c->d_rho, 0, nn * 8, c->stream);
  cudaMemsetAsync(&c->d_ps->bmean, 0, sizeof(double), c->stream);
  const double rtol = c->cfg.poisson_rtol;
  c->cfg.poisson_rtol = 1e-10;
  const pic_status st = poisson_solve(c, true);
  c->cfg.poisson_rtol = rtol;
  cudaMemcpyAsync(c->d_phiL, c->d_phi, nn * 8, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(c->d_phi, save_phi, nn * 8, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(c->d_rho, save_rho, nn * 8, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(c->d_ps, &ps_save, sizeof(ps_save), cudaMemcpyHostToDevice, c->stream);
  c->seen_solves = ps_save.n_solves;
  c->seen_outer = ps_save.sum_outer;
  c->seen_total = ps_save.sum_total;
  // the solve's residual passes wrote the empty box's field: back to the restored potential's
  launch_field(c);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
  return st;
}

pic_status learned_input(pic_ctx *c, int hpad, float *x, double *scale) {
  const int nn = c->g.nxn * c->g.nyn;
  if (hpad < c->g.nxn) return PIC_EINVAL;
  unsigned int *smax = reinterpret_cast<unsigned int *>(c->red.ticket) + 8;   // spare word
  cudaMemsetAsync(smax, 0, 4, c->stream);
  launch(k_absmax, c->red.nblocks, kThreads, 0, c->stream, c->d_rho, nn, smax);
  launch(k_learned_input, c->red.nblocks, kThreads, 0, c->stream, c->d_rho, c->d_nodeflags, c->g.nxn,
                                                                c->g.nyn, hpad, smax, x);
  unsigned int bits = 0;
  if (cudaMemcpyAsync(&bits, smax, 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return PIC_ECUDA;
  float f;
  std::memcpy(&f, &bits, 4);
  *scale = std::max(double(f), 1e-30);
  return PIC_OK;
}

pic_status learned_target(pic_ctx *c, int hpad, double scale, float *t) {
  const int nn = c->g.nxn * c->g.nyn;
  if (hpad < c->g.nxn || !(scale > 0)) return PIC_EINVAL;
  const pic_status st = ensure_vacuum_potential(c);
  if (st != PIC_OK) return st;
  launch(k_learned_target, c->red.nblocks, kThreads, 0, c->stream, c->d_phi, c->d_phiL, nn,
         hpad * c->g.nyn, 1.0 / scale, t);
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

// The learned initial guess inside the step, all on the device: s = max |rho|,
// the network's input, its forward pass, phi = phi_L + s y on the free nodes.
cudaError_t launch_learned_guess(pic_ctx *c) {
  const int nn = c->g.nxn * c->g.nyn;
  const int hpad = unet_height(c->net);
  unsigned int *smax = reinterpret_cast<unsigned int *>(c->red.ticket) + 8;   // spare word
  cudaMemsetAsync(smax, 0, 4, c->stream);
  launch(k_absmax, c->red.nblocks, kThreads, 0, c->stream, c->d_rho, nn, smax);
  launch(k_learned_input, c->red.nblocks, kThreads, 0, c->stream, c->d_rho, c->d_nodeflags, c->g.nxn,
         c->g.nyn, hpad, smax, c->d_net_x);
  unet_forward_only(c->net, c->d_net_x);
  launch(k_guess_learned_dev, c->red.nblocks, kThreads, 0, c->stream, c->d_phi, c->d_phiL, c->d_nodeflags,
         unet_output(c->net), smax, nn);
  c->launches += 3 + unet_forward_kernels();
  return cudaGetLastError();
}

pic_status poisson_with_guess(pic_ctx *c, int guess, const float *y, double scale, double *stats) {
  const int nn = c->g.nxn * c->g.nyn;
  if (guess >= 2) {
    const pic_status st = ensure_vacuum_potential(c);
    if (st != PIC_OK) return st;
  }
  cudaEventRecord(c->tev[0], c->stream);
  if (guess == 2)
    cudaMemcpyAsync(c->d_phi, c->d_phiL, size_t(nn) * 8, cudaMemcpyDeviceToDevice, c->stream);
  if (guess == 3) {
    if (!y) return PIC_EINVAL;
    launch(k_guess_learned, c->red.nblocks, kThreads, 0, c->stream, c->d_phi, c->d_phiL, c->d_nodeflags,
                                                                  y, scale, nn);
  }
  const pic_status st = poisson_solve(c, guess == 0);
  cudaEventRecord(c->tev[1], c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->tev[0], c->tev[1]);
  if (stats) {
    stats[0] = c->h_ps->total_iters;
    stats[1] = c->h_ps->outer_iters;
    stats[2] = c->h_ps->rel;
    stats[3] = ms;
  }
  return st;
}

}  // namespace picgb
