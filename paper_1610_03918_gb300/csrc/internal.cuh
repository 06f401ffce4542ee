// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "picgb.h"

namespace picgb {

// Fixed-point deposit: one particle's CIC shares are quantised to 2^-20 of
// its weight, three shares rounded to nearest-even and the fourth the
// remainder, so each particle deposits exactly 2^20 units.
constexpr int kFracBits = 20;
constexpr uint32_t kQ = 1u << kFracBits;

// Particle tiles: a sorted tile's particles are processed by one CTA with
// the field and the deposit of a window (tile + halo) held in shared memory.
// The tile shape (powers of two, in cells), the halo and the CTA size form a
// variant of the particle store, chosen per run by the autotuner
// (pic_autotune); results do not depend on it.
struct TileVariant {
  int log2x, log2y;   // tile of 2^log2x x 2^log2y cells
  int halo;           // window = tile + halo cells on every side
  int threads;        // CTA size of the particle kernel
};
constexpr int kNumTileVariants = 4;
constexpr TileVariant kTileVariants[kNumTileVariants] = {
    {4, 4, 4, 128},    // 16 x 16
    {5, 4, 4, 128},    // 32 (x) x 16 (y)
    {4, 5, 4, 128},    // 16 (x) x 32 (y)
    {5, 5, 4, 256},    // 32 x 32
};
constexpr int kMinTileLog2 = 4;  // the smallest tile (16 x 16) sizes the tile arrays
constexpr int kChunk = 4092;     // particles per work item (multiple of 4, <= 4095)
constexpr int kWalkLimit = 16;   // face crossings followed per move

// Double-float values.  The potential, the charge density and the Dirichlet
// data are held on the device as unevaluated sums hi + lo of two floats
// (float2: x = hi, y = lo, |lo| <= ulp(hi) / 2), about 48 significant bits,
// so the field-side kernels run on the FP32 pipes.  The sums are built from
// the error-free transformations TwoSum (Knuth) and Fast2Sum (Dekker) and
// the product from the FMA-based TwoProduct; the pair addition is the
// accurate double-double addition of Hida, Li and Bailey (2001).  Every
// operation is an explicitly rounded intrinsic, so nothing is contracted or
// reassociated by the compiler.
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv)));
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  float2 s = two_sum(a.x, b.x);
  const float2 t = two_sum(a.y, b.y);
  s = fast_two_sum(s.x, __fadd_rn(s.y, t.x));
  return fast_two_sum(s.x, __fadd_rn(s.y, t.y));
}
__device__ __forceinline__ float2 pair_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 pair_sub(float2 a, float2 b) { return pair_add(a, pair_neg(b)); }
// pair + float
__device__ __forceinline__ float2 pair_add_f(float2 a, float b) {
  const float2 s = two_sum(a.x, b);
  return fast_two_sum(s.x, __fadd_rn(s.y, a.y));
}
__device__ __forceinline__ float2 pair_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return fast_two_sum(p, e);
}
// a signed 64-bit integer, exactly when |x| < 2^48: x = h 2^24 + l with
// 0 <= l < 2^24, both parts exact floats, joined by TwoSum
__device__ __forceinline__ float2 pair_from_ll(long long x) {
  const int h = int(x >> 24);
  const int l = int(x & 0xffffff);
  return two_sum(__fmul_rn(__int2float_rn(h), 16777216.f), __int2float_rn(l));
}
// conversions to and from FP64 (host side, and rare device paths)
__host__ __device__ inline float2 pair_split(double d) {
  const float h = float(d);
  return make_float2(h, float(d - double(h)));
}
__host__ __device__ inline double pair_join(float2 p) { return double(p.x) + double(p.y); }

// Step phases timed by events: sort | particle kernel | rho | Poisson solve
// (with the field), bounded by kPhaseEvents events.
constexpr int kPhaseEvents = 5;
constexpr int kTimeSlots = 64;

// Division by a divisor fixed at set-up, by a multiply-high and shifts on the
// integer pipes (Granlund and Montgomery, PLDI 1994): for 1 <= d < 2^31 and
// 0 <= n < 2^31, with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// t = hi32(m n) and n / d = (t + ((n - t) >> 1)) >> (l - 1); d = 1 passes n.
struct FastDiv {
  uint32_t d, m, l;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.l = 0;
  while ((uint64_t(1) << f.l) < d) ++f.l;
  f.m = d <= 1 ? 0u : uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << f.l) - d)) / d + 1);
  return f;
}
__host__ __device__ __forceinline__ int fdiv(int n, const FastDiv &f) {
  if (f.d == 1) return n;
#ifdef __CUDA_ARCH__
  const uint32_t t = __umulhi(f.m, uint32_t(n));
#else
  const uint32_t t = uint32_t((uint64_t(f.m) * uint32_t(n)) >> 32);
#endif
  return int((t + ((uint32_t(n) - t) >> 1)) >> (f.l - 1));
}

struct Geom {
  int nx, ny;          // cells
  int px, py;          // periodic flags
  int nxn, nyn;        // nodes
  int ntx, nty;        // tiles of the tile variant in use
  int tsx, tsy;        // its tile shape: 2^tsx x 2^tsy cells
  FastDiv dnyn;        // division by nyn (node index -> row)
};

// Cell mask bits (uint8 per cell)
constexpr uint8_t kCellPlasma = 1;
constexpr uint8_t kCellInterior = 2;   // the cell and its eight neighbours are plasma

// Node flag bits (uint8 per node)
constexpr uint8_t kFree = 1;     // not a Dirichlet node
constexpr uint8_t kOpenXm = 2;   // edge (i-1, j) - (i, j) borders a plasma cell
constexpr uint8_t kOpenXp = 4;   // edge (i, j) - (i+1, j)
constexpr uint8_t kOpenYm = 8;   // edge (i, j-1) - (i, j)
constexpr uint8_t kOpenYp = 16;  // edge (i, j) - (i, j+1)

struct ParticleBuf {
  int32_t *cell;
  float *fx, *fy, *vx, *vy;
  uint32_t *id;
};

struct Chunk {
  int32_t species, tile, begin, end;
};
static_assert(sizeof(Chunk) == 16, "a chunk is written as one 16-byte vector");

// device pointers of up to 64 ranks' exchange buffers (by value, as a kernel argument)
struct DevPtrs {
  unsigned long long *p[64];
};

// Device-side scalars of one Poisson solve.
struct PoissonState {
  double bb;          // ||b||^2
  double rr64;        // ||b - A phi||^2 (outer: the certificate)
  double rel;         // sqrt(rr64 / bb)
  double rel_first;   // rel of the initial guess (the solve's first checking pass)
  double bmean;       // mean of b (doubly periodic box only)
  double rz, rz_old, rr, rr0;       // inner PCG: gamma = <r, z>, its previous value, ||r||^2
  double delta;                      // <z, A z>
  double alpha, beta;
  double alpha_next, beta_next;      // the coefficients of the next CG update
  float cg_f[3];                     // alpha_next, beta_next, zmean in FP32
  double zmean;
  double tol_in;      // inner target relative to the inner initial residual
  int32_t inner_done, outer_done;
  int32_t inner_iters, total_iters;
  int32_t outer_iters, go;   // go: the last residual check asked for another inner solve
  // running totals over all solves (never reset): solves ended, their outer
  // passes and inner iterations, for the launch count of timed graph steps
  long long n_solves, sum_outer, sum_total;
};

struct MGLevel {
  int nx, ny, nxn, nyn;
  float h2;            // squared mesh spacing (4^level)
  uint8_t *free;       // level 0: 1 = unknown, 0 = Dirichlet (zero correction)
  uint16_t *sid;       // levels >= 1: 0 = not an unknown, k = stencil k-1 of stab
  float *stab;         // levels >= 1: unique Galerkin 9-point stencils [k][3x3]
  int nst;             // number of unique stencils
  float *u, *f;        // correction and right-hand side
  float *upre = nullptr;   // levels above lc: u after the pre-smoothing
};

struct Reducer {
  double *part;        // per-block partials
  unsigned int *ticket;
  int nblocks;
};

// Direct inner solve of the Poisson correction equation for boxes periodic in
// y (ny a power of two) and bounded in x whose free nodes are the full rows
// 1..m plus, optionally, one interface row xs = m + 1 and a slot below it
// sharing the interface's columns [c0, c0 + wc): the trench and the plates.
// Rows 1..m: FFT along y, then per Fourier mode k the tridiagonal system
// tridiag(-1, 4 - 2 cos(2 pi k / ny), -1) along x by parallel cyclic
// reduction.  Slot rows xs+1..xs+ms: sine transform across its wc columns,
// one tridiagonal system per sine mode along x.  The interface values come from
// the wc x wc Schur complement of the coupled system (precomputed inverse).
struct FastPoisson {
  int enabled = 0;
  int ny = 0, nk = 0, logny = 0;   // FFT size, modes ny / 2 + 1
  int m = 0, xs = 0;               // rectangle rows 1..m, interface row xs
  int slot = 0;                    // interface and slot present
  int c0 = 0, wc = 0, ms = 0;      // slot columns [c0, c0 + wc), rows xs+1 .. xs+ms
  float2 *tw = nullptr;            // [ny] exp(-2 pi i t / ny)
  float *dk = nullptr;             // [nk] diagonal of each slab mode's system
  float *z = nullptr;              // [m][nk] column m of the inverse tridiagonal (interface response)
  float2 *vhat = nullptr;          // [m][nk] spectra of the rows
  float *phi = nullptr;            // [wc][wc] orthonormal sine basis of the slot, [mode][column]
  float2 *twc = nullptr;          // [wc][nk] inverse-DFT weights of the interface columns
  float2 *fh = nullptr;           // [nk] spectrum of the interface values
  float *sh = nullptr;            // [wc] sine spectrum of the interface values
  float *sb = nullptr;             // [wc] diagonal of each slot sine mode's system
  float *zs = nullptr;             // [wc][ms] slot responses to a unit first-row value
  float *sinv = nullptr;           // [wc][wc] inverse of the interface Schur complement
  float *vs = nullptr;             // [wc][ms] solved slot spectra
  float *ug = nullptr;             // [wc] interface values
  int kernels = 0;                 // launches per inner solve
};

// Programmatic dependent launch.  The solver's kernels wait for the grid
// before them (its results are then visible) and at once let the next kernel
// of the stream be scheduled, so that kernel's blocks are resident and waiting
// when this one ends instead of being launched only then.  Both instructions
// are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory");
}

#ifndef PICGB_NO_PDL
constexpr bool kPdl = true;
#else
constexpr bool kPdl = false;
#endif

template <typename... P, typename... A>
void launch(void (*k)(P...), int grid, int block, size_t smem, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(block));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &at;
  cfg.numAttrs = kPdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, args...);
}

}  // namespace picgb

struct pic_ctx {
  pic_config cfg;
  picgb::Geom g;
  int dev;
  int num_sms;
  cudaStream_t stream;
  bool own_stream;

  // geometry
  int src_x0, src_x1;       // ion recycling source rows [src_x0, src_x1)
  uint8_t *d_cellmask;      // [nx*ny] 1 = plasma
  uint8_t *d_nodeflags;     // [nxn*nyn]
  float *d_lift;            // [nxn*nyn] sum of Dirichlet neighbour values (free nodes; norms only)
  float2 *d_g;              // [nxn*nyn] Dirichlet values (0 at free nodes), double-float
  std::vector<uint8_t> h_nodeflags;
  std::vector<double> h_g;
  std::vector<uint8_t> h_electrode;   // [nxn*nyn] node held at the electrode potential
  // RF bias (phi_rf_amp != 0): the electrode's Dirichlet nodes with their
  // static values, and the free nodes next to them with their count of such
  // neighbours and their static lift
  int n_rf_dir, n_rf_lift;
  int32_t *d_rf_dir;
  float2 *d_rf_g0;
  int32_t *d_rf_lift;
  float *d_rf_cnt, *d_rf_lift0;

  // fields
  unsigned long long *d_acc;   // [2][nnodes] fixed-point species weights, then (exchange
                               // buffer of a decomposed run) the bottom counts [2][ny]
  int phase;                   // decomposed run: 0 idle, 1 prepare / 2 step particle phase done
  // double-float (hi, lo) node arrays
  float2 *d_rho_ext;
  float2 *d_rho;               // net charge density
  float2 *d_phi;               // the potential (Dirichlet values included)
  float2 *d_phi_prev;          // potential of the previous step (extrapolated warm start)
  float2 *d_phiL;              // potential of the empty box (learned warm start), lazily
  pic_unet *net;               // warm-start network of this context (warm_start 3), owned
  float *d_net_x;              // its input [hpad][nyn][2]
  float2 *d_E;
  double *d_fe;                // [2]: field energy of E just computed, of E used by last step

  // Poisson
  int nlev, lc;                // levels, first level solved by the single-CTA kernel
  std::vector<picgb::MGLevel> lev;
  float *d_r32, *d_z, *d_p, *d_w, *d_q, *d_e;   // inner PCG vectors (w = A z)
  size_t coarse_smem;          // dynamic shared memory of the single-CTA coarse V-cycle
  int ncoarse;                 // unknowns of the coarsest level (dense inverse), 0 = sweeps
  float *d_cinv;
  int *d_cidx;
  picgb::PoissonState *d_ps;
  picgb::PoissonState *h_ps;   // pinned mirror
  picgb::Reducer red;
  int singular;
  picgb::FastPoisson fp;       // direct inner solve (enabled when the geometry allows it)
  double last_ms;
  int last_outer;
  cudaEvent_t ev0, ev1;

  // particles
  picgb::ParticleBuf pb[2][2];
  int cur[2];                  // host mirror of d_cur
  picgb::ParticleBuf *d_pbufs; // [species][2] on the device
  int32_t *d_cur;              // current buffer per species (device)
  int64_t cap[2];              // slots allocated per buffer
  int needs_sort;
  int pending_kick[2];
  int steps_since_sort;
  // Sort interval tuning (cfg.sort_every = 0): after one sort the particle
  // kernel is timed for kTuneSteps steps, then the interval S minimising
  // (sort time + particle time of the S steps after a sort) / S is kept.
  int tune_state;              // 0 not started, 1 measuring, 2 chosen
  int sort_interval;           // the chosen S
  float tune_sort_ms;
  std::vector<float> tune_particle_ms;
  uint32_t *d_tile_count;      // [2][ntiles]
  uint32_t *d_tile_cursor;     // [2][ntiles]
  uint32_t *d_tile_start;      // [2][ntiles]
  picgb::Chunk *d_chunks;
  int32_t *d_nchunks;
  int64_t max_chunks;
  int tile_variant;            // index into kTileVariants
  int suppress_sort;           // autotuning: no scheduled sorts while a variant is timed
  int max_tiles;               // tiles of the smallest tile shape (array sizes)
  int64_t *d_nslots;           // [4]: slots in use per species; [2..3] staged by the sort
  double *d_ke_part;           // [max_chunks]
  int32_t *d_step;

  // tallies and status
  unsigned long long *d_walls;    // [2][8]
  unsigned long long *d_bottom;   // [2][ny]
  pic_hit *d_hits;
  unsigned long long *d_nhits;
  uint32_t *d_status;
  uint32_t *h_status;             // pinned

  // staging for pic_load / diag
  double *d_stage;
  double *d_diag;                 // per-block partials of the particle moments
  int64_t stage_n;
  int fields_dirty;
  int64_t step;
  // captured step graphs [with the tile sort][with phase event nodes]
  cudaGraph_t graph[2][2];
  cudaGraphExec_t gexec[2][2];
  // decomposed run: particle phase without / with the sort, field phase
  cudaGraph_t graph_dp[3];
  cudaGraphExec_t gexec_dp[3];
  cudaGraphNode_t evnode[2][picgb::kPhaseEvents];   // event nodes of the [.][1] graphs
  // per-phase timing (PIC_DIAG_TIMING): each timed step records its phase
  // boundaries into its own slot of the pool, read back when the pool is full
  // or a diagnostic is read, so timed steps are not serialised with the host
  cudaEvent_t tev[picgb::kPhaseEvents];              // capture placeholders, solve timing
  cudaEvent_t tpool[picgb::kTimeSlots][picgb::kPhaseEvents];
  int tpend;                                         // slots recorded, not yet read
  uint8_t tslot_tune[picgb::kTimeSlots];             // the slot's step feeds the sort tuning
  long long seen_solves, seen_outer, seen_total;     // solve totals already counted
  double t_part, t_sort, t_poisson, t_other;
  int64_t t_steps, t_sorts, launches, t_slots;
  std::vector<void *> allocs;
};

namespace picgb {

// api.cu
void *dev_alloc(pic_ctx *c, size_t bytes);
// a temporary device buffer through the context's allocator (released by tmp_free)
void *tmp_alloc(pic_ctx *c, size_t bytes);
void tmp_free(pic_ctx *c, void *p);
// records "where: CUDA error string" as the calling thread's last error; returns e
cudaError_t note(cudaError_t e, const char *where);

// particles.cu
cudaError_t launch_sort(pic_ctx *c);
// switches the particle store to tile variant v (the next step must sort)
void set_tile_variant(pic_ctx *c, int v);
// mode 0: full step; 1: deposit only; 2: kick only (factor * dt, flagged species)
cudaError_t launch_particles(pic_ctx *c, int mode, float kick_factor, const int *species_mask);
cudaError_t launch_load_convert(pic_ctx *c, int s, const double *d_x, const double *d_y,
                                const double *d_vx, const double *d_vy, const uint32_t *d_id,
                                int64_t offset, int64_t n);
cudaError_t launch_export_state(pic_ctx *c, int s, double *d_out, int64_t n_live,
                                unsigned long long *d_counter);
// live particles of species s in stored form, compacted into out (checkpoints)
cudaError_t launch_export_raw(pic_ctx *c, int s, ParticleBuf out, int64_t cap,
                              unsigned long long *d_counter);
// per-block partials [sum vx, sum vy, live] of species s into d_part[3 * nblocks]
cudaError_t launch_moments(pic_ctx *c, int s, double *d_part, int nblocks);

// poisson.cu
cudaError_t poisson_setup(pic_ctx *c);
// Direct inner solve (fastpoisson.cu): set-up when the geometry allows it
// (leaves c->fp.enabled = 0 otherwise) and the launches that turn the FP32
// residual r into the correction e.
cudaError_t fast_poisson_setup(pic_ctx *c);
void fast_poisson_launch(pic_ctx *c, const float *r, float2 *pot, PoissonState *ps);
cudaError_t launch_rho(pic_ctx *c, int advance_step, int init_solve = 0);
// In a captured step with the direct solve and the previous potential as the
// guess, the solve's first residual pass forms rho itself (no density kernel).
bool rho_in_solve(const pic_ctx *c);
pic_status poisson_solve(pic_ctx *c, bool zero_guess);
cudaError_t poisson_capture(pic_ctx *c, cudaGraph_t top, std::vector<cudaGraphNode_t> &deps);
int64_t poisson_kernel_count(pic_ctx *c, int64_t S, int64_t O, int64_t I);
pic_status ensure_vacuum_potential(pic_ctx *c);
pic_status learned_input(pic_ctx *c, int hpad, float *x, double *scale);
pic_status poisson_with_guess(pic_ctx *c, int guess, const float *y, double scale, double *stats);
cudaError_t launch_field(pic_ctx *c);
// learned warm start inside the step: absmax of rho, network input, network,
// guess phi = phi_L + s y on the free nodes (device-side scale)
cudaError_t launch_learned_guess(pic_ctx *c);
pic_status learned_target(pic_ctx *c, int hpad, double scale, float *t);

// conv_tc.cu: one 3x3 convolution on the tcgen05 tensor cores (BF16 NHWC,
// FP32 accumulation, bias and optional ReLU)
struct ConvTC {
  const __nv_bfloat16 *in;
  int in_cs, in_off, cin;
  const __nv_bfloat16 *w;     // [cout][9][cin]
  const float *bias;          // [cout] or null
  __nv_bfloat16 *out;
  int out_cs, out_off, cout;
  int B, H, W;
  int relu;
  int *err;                   // device error word (a bounded wait gave up)
  // transposed 2x2 stride-2 convolution instead (up_cout > 0): w is
  // [4 up_cout][cin] (row (2a + c) up_cout + co), H x W the input's size,
  // out 2H x 2W; this launch computes the cout GEMM columns from n_base
  int up_cout = 0;
  int n_base = 0;
};
bool conv3x3_tc_supported(int cin, int cout, int in_cs, int in_off, int out_cs, int out_off, int W);
cudaError_t conv3x3_tc(const ConvTC &c, cudaStream_t s);
// sets the kernels' shared-memory attributes (before any stream capture)
cudaError_t conv3x3_tc_prepare();
// data gradient of the 2x2 stride-2 transposed convolution on the tensor
// cores: in = its output gradient [B][2H][2W][in_cs] (channels in_off ..
// in_off + cin), w = BF16 [4 cout][cin] (row (2a + c) cout + ci: the master
// weights' own order), out = the gradient at its input [B][H][W] (cout
// channels from out_off in rows of out_cs)
cudaError_t conv_upback_tc(const ConvTC &c, cudaStream_t s);
// weight gradient of a 3x3 convolution on the tensor cores:
// dw[co][3 dy + dx][ci] += sum over pixels p of dpre[p][co] in[p + (dy - 1, dx - 1)][in_off + ci]
// (zero padding); dpre [B][H][W][cout] contiguous, in [B][H][W][in_cs]; FP32
// atomic adds.  cout 32 or a multiple of 64, cin 16, 32 or a multiple of 64,
// dw 16-byte aligned.
struct WgradTC {
  const __nv_bfloat16 *dpre, *in;
  int in_cs, in_off, cin, cout;
  float *dw;
  int B, H, W;
  int *err;                   // device error word (a bounded wait gave up)
};
bool conv_wgrad_tc_supported(int cin, int cout, int in_cs, int in_off, const float *dw);
cudaError_t conv_wgrad_tc(const WgradTC &g, cudaStream_t s);
// weight gradient of the 2x2 stride-2 transposed convolution on the tensor
// cores: dw[a][c][ci][co] += sum over input pixels (y, x) of
// in[y][x][ci] g[2y + a][2x + c][g_off + co]; in [B][H][W][cin] contiguous,
// g [B][2H][2W][g_cs]; FP32 atomic adds.  cin a multiple of 64, cout 32 or a
// multiple of 64.
struct UpWgradTC {
  const __nv_bfloat16 *in, *g;
  int cin, g_cs, g_off, cout;
  float *dw;
  int B, H, W;
  int *err;
};
bool conv_upwgrad_tc_supported(int cin, int cout, int g_cs, int g_off);
cudaError_t conv_upwgrad_tc(const UpWgradTC &g, cudaStream_t s);
// the network's first 3x3 convolution (2 FP32 input channels per pixel ->
// 32 BF16 outputs [p][32]) on the tensor cores; w: BF16 [32][9][wcin]
cudaError_t conv_in_tc(const float2 *x, const __nv_bfloat16 *w, int wcin, const float *bias,
                       __nv_bfloat16 *out, int B, int H, int W, int relu, int *err, cudaStream_t s);

// unet.cu
void unet_forward_only(pic_unet *u, const float *x);
const float *unet_output(const pic_unet *u);
int unet_height(const pic_unet *u);
int unet_width(const pic_unet *u);
int unet_batch(const pic_unet *u);
int unet_forward_kernels();
pic_status unet_copy_params(pic_unet *dst, const pic_unet *src);
// RF bias: the electrode's Dirichlet values (in phi and in the Dirichlet
// data) and the lift at t = (step + advance) dt; no-op without RF
cudaError_t launch_rf_bias(pic_ctx *c, int advance);

}  // namespace picgb
