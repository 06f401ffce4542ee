// Particle-side kernels: tile counting sort, the fused gather / leapfrog
// push / absorption / cloud-in-cell deposit kernel, and state conversion.
//
// Particles are stored per species as structure-of-arrays: int32 cell
// index packed as (i << 16) | j (-1 = dead or padding), FP32 offsets fx, fy in [0, 1)
// inside the cell, FP32 velocities vx, vy (at half steps), uint32 id.
// Every sort_every steps they are counting-sorted by 16x16-cell tile; each
// tile's segment is padded to a multiple of 4 slots so that one thread moves
// four particles with 16-byte vector loads and stores.
#include <cuda_runtime.h>

#include "internal.cuh"
#include "philox.cuh"

namespace picgb {
namespace {

__device__ __forceinline__ int wrapmod(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

__device__ __forceinline__ int cell_i(int c) { return c >> 16; }
__device__ __forceinline__ int cell_j(int c) { return c & 0xffff; }
__device__ __forceinline__ int pack_cell(int i, int j) { return (i << 16) | j; }

__device__ __forceinline__ int tile_of(const Geom &g, int c) {
  return (cell_i(c) >> g.tsx) * g.nty + (cell_j(c) >> g.tsy);
}

// ---------------------------------------------------------------------------
// Counting sort by tile
// ---------------------------------------------------------------------------
constexpr int kHistSmemTiles = 12288;   // shared-memory tile histogram up to 48 KB

struct SortArgs {
  const ParticleBuf *pbufs;  // [species][2] on the device
  int32_t *cur;              // current buffer per species (device)
  const int64_t *nslots;   // slots in use in src, per species
  uint32_t *count, *cursor, *start;   // [2][ntiles]
  Chunk *chunks;
  int32_t *nchunks;
  int64_t *nslots_out;
  Geom g;
  int ntiles;
};

// The counting passes take 4 consecutive slots per lane (16-byte loads, 128
// slots per warp per iteration) and treat them as 4 independent groups, so a
// warp has all its loads, then 4 match / atomic rounds, in flight at once.
// Slot counts are multiples of 4 within the buffers' capacity, so a vector
// read starting below n stays inside the allocation; slots >= n are ignored.
// Tile histogram.  Each block takes a contiguous range of slots, so its
// particles fall in a few tiles (they were sorted a few steps ago); with SMEM
// the counts gather in a shared-memory histogram and only its nonzero bins
// reach the global counters, instead of every warp's atomics meeting on the
// same few hot counters.
template <bool SMEM>
__global__ void k_sort_hist(SortArgs a) {
  extern __shared__ uint32_t hist[];
  const int s = blockIdx.y;
  const int64_t n = a.nslots[s];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  uint32_t *cnt = a.count + int64_t(s) * a.ntiles;
  uint32_t *h = SMEM ? hist : cnt;
  if (SMEM) {
    for (int t = threadIdx.x; t < a.ntiles; t += blockDim.x) hist[t] = 0u;
    __syncthreads();
  }
  const int32_t *cell = a.pbufs[2 * s + a.cur[s]].cell;
  const int64_t units = (n + 127) / 128;                 // 128 slots per warp step
  const int64_t per = (units + gridDim.x - 1) / gridDim.x;
  const int64_t u1 = min(units, int64_t(blockIdx.x + 1) * per);
  for (int64_t u = int64_t(blockIdx.x) * per + wib; u < u1; u += nwb) {
    const int64_t p = u * 128 + 4 * lane;
    int4 c4 = make_int4(-1, -1, -1, -1);
    if (p < n) c4 = *reinterpret_cast<const int4 *>(cell + p);
    const int cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = (p + j < n && cc[j] >= 0) ? tile_of(a.g, cc[j]) : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, t);
      if (t >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[t], (uint32_t)__popc(peers));
    }
  }
  if (SMEM) {
    __syncthreads();
    for (int t = threadIdx.x; t < a.ntiles; t += blockDim.x)
      if (hist[t]) atomicAdd(&cnt[t], hist[t]);
  }
}

// Block-wide exclusive scan of one value per thread (blockDim == 1024).
__device__ uint32_t block_exscan(uint32_t v, uint32_t *total) {
  __shared__ uint32_t warp_sums[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  const uint32_t before = (w > 0 ? warp_sums[w - 1] : 0u) + x - v;
  *total = warp_sums[31];
  __syncthreads();
  return before;
}

// One CTA of 1024 threads: tile starts (padded to 4 slots), the chunk work
// list of both species, padding slots marked dead, counters reset.  The chunk
// list is written with consecutive threads on consecutive chunks: each thread
// finds the tile of its chunk by a binary search over the tiles' first chunk
// indices, kept in shared memory.
__global__ void __launch_bounds__(1024) k_sort_scan(SortArgs a) {
  __shared__ uint32_t s_first[1025];   // first chunk of each tile of the round, then the round's total
  __shared__ uint32_t s_off[1024], s_padded[1024];
  uint32_t chunk_base = 0;
  for (int s = 0; s < 2; ++s) {
    uint32_t slot_base = 0;
    uint32_t *cnt = a.count + int64_t(s) * a.ntiles;
    uint32_t *cur = a.cursor + int64_t(s) * a.ntiles;
    uint32_t *st = a.start + int64_t(s) * a.ntiles;
    int32_t *dcell = a.pbufs[2 * s + (a.cur[s] ^ 1)].cell;
    for (int t0 = 0; t0 < a.ntiles; t0 += 1024) {
      const int t = t0 + threadIdx.x;
      uint32_t n = 0, padded = 0, nch = 0;
      if (t < a.ntiles) {
        n = cnt[t];
        padded = (n + 3u) & ~3u;
        nch = (padded + kChunk - 1) / kChunk;
      }
      uint32_t tot_slots, tot_ch;
      const uint32_t off = block_exscan(padded, &tot_slots) + slot_base;
      const uint32_t first = block_exscan(nch, &tot_ch);
      s_first[threadIdx.x] = first;
      s_off[threadIdx.x] = off;
      s_padded[threadIdx.x] = padded;
      if (threadIdx.x == 0) s_first[1024] = tot_ch;
      if (t < a.ntiles) {
        st[t] = off;
        cur[t] = 0;
        cnt[t] = 0;
        for (uint32_t k = n; k < padded; ++k) dcell[off + k] = -1;
      }
      __syncthreads();
      for (uint32_t c = threadIdx.x; c < tot_ch; c += 1024) {
        // the last tile k of the round with first[k] <= c (it has at least one chunk)
        int lo = 0, hi = 1024;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (s_first[mid] <= c) lo = mid; else hi = mid;
        }
        const uint32_t q = c - s_first[lo];
        const uint32_t b0 = s_off[lo] + q * kChunk;
        const uint32_t b1 = s_off[lo] + min(s_padded[lo], (q + 1) * kChunk);
        reinterpret_cast<int4 *>(a.chunks)[chunk_base + c] = make_int4(s, t0 + lo, int(b0), int(b1));
      }
      __syncthreads();
      slot_base += tot_slots;
      chunk_base += tot_ch;
    }
    if (threadIdx.x == 0) a.nslots_out[s] = slot_base;   // published by k_sort_finish
  }
  if (threadIdx.x == 0) *a.nchunks = int32_t(chunk_base);
}

__global__ void k_sort_finish(int64_t *nslots, int32_t *cur) {
  nslots[0] = nslots[2];
  nslots[1] = nslots[3];
  cur[0] ^= 1;
  cur[1] ^= 1;
}

__global__ void k_sort_scatter(SortArgs a) {
  const int s = blockIdx.y;
  const int64_t n = a.nslots[s];
  const int lane = threadIdx.x & 31;
  const unsigned lower = (1u << lane) - 1u;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  uint32_t *cur = a.cursor + int64_t(s) * a.ntiles;
  const uint32_t *st = a.start + int64_t(s) * a.ntiles;
  const ParticleBuf S = a.pbufs[2 * s + a.cur[s]], D = a.pbufs[2 * s + (a.cur[s] ^ 1)];
  for (int64_t base = warp * 128; base < n; base += nwarps * 128) {
    const int64_t p = base + 4 * lane;
    int4 c4 = make_int4(-1, -1, -1, -1);
    float4 fx4 = make_float4(0.f, 0.f, 0.f, 0.f), fy4 = fx4, vx4 = fx4, vy4 = fx4;
    uint4 id4 = make_uint4(0u, 0u, 0u, 0u);
    if (p < n) {
      c4 = *reinterpret_cast<const int4 *>(S.cell + p);
      fx4 = *reinterpret_cast<const float4 *>(S.fx + p);
      fy4 = *reinterpret_cast<const float4 *>(S.fy + p);
      vx4 = *reinterpret_cast<const float4 *>(S.vx + p);
      vy4 = *reinterpret_cast<const float4 *>(S.vy + p);
      id4 = *reinterpret_cast<const uint4 *>(S.id + p);
    }
    const int cc[4] = {c4.x, c4.y, c4.z, c4.w};
    const float fx[4] = {fx4.x, fx4.y, fx4.z, fx4.w}, fy[4] = {fy4.x, fy4.y, fy4.z, fy4.w};
    const float vx[4] = {vx4.x, vx4.y, vx4.z, vx4.w}, vy[4] = {vy4.x, vy4.y, vy4.z, vy4.w};
    const uint32_t id[4] = {id4.x, id4.y, id4.z, id4.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = (p + j < n && cc[j] >= 0) ? tile_of(a.g, cc[j]) : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, t);
      const int leader = __ffs(peers) - 1;
      uint32_t b = 0;
      if (t >= 0 && lane == leader) b = atomicAdd(&cur[t], (uint32_t)__popc(peers));
      b = __shfl_sync(0xffffffffu, b, leader);
      if (t >= 0) {
        const int64_t d = int64_t(st[t]) + b + __popc(peers & lower);
        D.cell[d] = cc[j];
        D.fx[d] = fx[j];
        D.fy[d] = fy[j];
        D.vx[d] = vx[j];
        D.vy[d] = vy[j];
        D.id[d] = id[j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Fused particle kernel
// ---------------------------------------------------------------------------
struct PArgs {
  const ParticleBuf *pbufs;  // [species][2] on the device
  const int32_t *cur;        // current buffer per species (device)
  const Chunk *chunks;
  const int32_t *nchunks;
  const float2 *E;
  unsigned long long *acc;   // [2][nnodes]
  const uint8_t *cellmask;
  Geom g;
  float qdt[2];              // alpha_s * dt (times the kick factor in kick mode)
  float dt;
  int kick[2];               // kick mode: species to kick
  unsigned long long *walls, *bottom;
  pic_hit *hits;
  unsigned long long *nhits;
  long long hit_cap;
  uint32_t *status;
  const int32_t *step;
  double *ke_part;
  double *fe;                // [0] energy of the current E, [1] of the E used by the last step
  // ion recycling: absorbed ions re-enter in cell rows [src_x0, src_x0 + src_rows)
  int recycle;
  int src_x0, src_rows;
  uint2 key;                 // Philox key (the seed)
  float vth_i;               // thermal speed of the re-entering ions
};

// The shared-memory window of a tile variant: tile + halo cells, +1 nodes.
template <int V>
struct Win {
  static constexpr int TX = 1 << kTileVariants[V].log2x;
  static constexpr int TY = 1 << kTileVariants[V].log2y;
  static constexpr int H = kTileVariants[V].halo;
  static constexpr int THREADS = kTileVariants[V].threads;
  static constexpr int WXc = TX + 2 * H;   // window cells
  static constexpr int WYc = TY + 2 * H;
  static constexpr int NWX = WXc + 1;      // window nodes
  static constexpr int NWY = WYc + 1;
};


__device__ __forceinline__ void deposit_global(const PArgs &a, unsigned long long *acc, int i,
                                               int j, int w00, int w01, int w10, int w11) {
  const Geom &g = a.g;
  int i1 = i + 1, j1 = j + 1;
  if (g.px && i1 == g.nxn) i1 = 0;
  if (g.py && j1 == g.nyn) j1 = 0;
  atomicAdd(&acc[i * g.nyn + j], (unsigned long long)(long long)w00);
  atomicAdd(&acc[i * g.nyn + j1], (unsigned long long)(long long)w01);
  atomicAdd(&acc[i1 * g.nyn + j], (unsigned long long)(long long)w10);
  atomicAdd(&acc[i1 * g.nyn + j1], (unsigned long long)(long long)w11);
}

// Fixed-point CIC shares.  Every rounding is spelled out (no contraction
// left to the compiler) so a particle's shares do not depend on the code
// path it took, and hence not on the particle order.  The fourth share is
// the remainder, so the four sum to exactly 2^20; it is -1 when the three
// rounded shares overshoot (a particle on a cell edge), which the window
// flush below accounts for.
__device__ __forceinline__ void cic_weights(float fx, float fy, int &w00, int &w01, int &w10,
                                            int &w11) {
  const float gx = __fsub_rn(1.0f, fx), gy = __fsub_rn(1.0f, fy);
  const float q = float(kQ);
  w00 = __float2int_rn(__fmul_rn(__fmul_rn(gx, gy), q));
  w10 = __float2int_rn(__fmul_rn(__fmul_rn(fx, gy), q));
  w01 = __float2int_rn(__fmul_rn(__fmul_rn(gx, fy), q));
  w11 = int(kQ) - w00 - w10 - w01;
}

// Bilinear interpolation of one component with explicit roundings.
__device__ __forceinline__ float bilerp(float fx, float fy, float gx, float gy, float e00,
                                        float e01, float e10, float e11) {
  const float lo = __fmaf_rn(fy, e01, __fmul_rn(gy, e00));
  const float hi = __fmaf_rn(fy, e11, __fmul_rn(gy, e10));
  return __fmaf_rn(fx, hi, __fmul_rn(gx, lo));
}

// Window-local coordinate of cell index i (window origin w0, period n when
// periodic).  The value is outside [0, W) when the cell is outside the window.
__device__ __forceinline__ int local_coord(int i, int w0, int n, int periodic) {
  int l = i - w0;
  if (periodic) l = l < 0 ? l + n : (l >= n ? l - n : l);
  return l;
}

template <int NWY>
__device__ __forceinline__ void deposit_shared(uint32_t *sAcc, int li, int lj, int w00, int w01,
                                               int w10, int w11) {
  const int k = li * NWY + lj;
  atomicAdd(&sAcc[k], (uint32_t)w00);
  atomicAdd(&sAcc[k + 1], (uint32_t)w01);
  atomicAdd(&sAcc[k + NWY], (uint32_t)w10);
  atomicAdd(&sAcc[k + NWY + 1], (uint32_t)w11);
}

// The rare path of a move: walk the crossed faces in order of the segment
// parameter (x face first on a tie).  The first face whose far cell is a
// conductor or outside a bounded direction absorbs the particle: its wall
// and bottom-cell tallies and a hit record are written and 1 is returned.
// A move longer than the walk limit is dropped (status bit, no tally) and 2
// is returned.  Otherwise the cell offset (oi, oj) of the end point is set
// and 0 returned.  Only particles in cells next to a wall or conductor, or
// moving more than one cell, come here.
__device__ __forceinline__ int walk_move(const PArgs &a, int s, int i, int j, float fx, float fy,
                                      float dx, float dy, int cx, int cy, float vx1, float vy1,
                                      const uint32_t *id, int64_t slot, int &oi, int &oj) {
  const Geom &g = a.g;
  const int si = cx > 0 ? 1 : -1, sj = cy > 0 ? 1 : -1;
  const float adx = fabsf(dx), ady = fabsf(dy);
  oi = 0;
  oj = 0;
  for (int k = 0; k < kWalkLimit; ++k) {
    const bool needx = oi != cx, needy = oj != cy;
    if (!needx && !needy) return 0;
    const float facex = float(si > 0 ? oi + 1 : oi);
    const float facey = float(sj > 0 ? oj + 1 : oj);
    const bool xfirst = __fmul_rn(fabsf(__fsub_rn(facex, fx)), ady) <=
                        __fmul_rn(fabsf(__fsub_rn(facey, fy)), adx);
    const bool takex = needx && (!needy || xfirst);
    if (takex) oi += si; else oj += sj;
    int gi = i + oi, gj = j + oj;
    bool outx = false, outy = false;
    if (g.px) gi = wrapmod(gi, g.nx); else outx = gi < 0 || gi >= g.nx;
    if (g.py) gj = wrapmod(gj, g.ny); else outy = gj < 0 || gj >= g.ny;
    if (outx || outy || !__ldg(&a.cellmask[gi * g.ny + gj])) {
      int wall, wcell;
      if (takex) {
        wall = si > 0 ? (outx ? PIC_WALL_XMAX : PIC_WALL_COND_PX)
                      : (outx ? PIC_WALL_XMIN : PIC_WALL_COND_MX);
        wcell = gj;
      } else {
        wall = sj > 0 ? (outy ? PIC_WALL_YMAX : PIC_WALL_COND_PY)
                      : (outy ? PIC_WALL_YMIN : PIC_WALL_COND_MY);
        wcell = gi;
      }
      atomicAdd(&a.walls[s * PIC_NWALLS + wall], 1ull);
      if (wall == PIC_WALL_XMAX) atomicAdd(&a.bottom[s * g.ny + wcell], 1ull);
      const unsigned long long h = atomicAdd(a.nhits, 1ull);
      if ((long long)h < a.hit_cap) {
        pic_hit rec;
        rec.id = id[slot];
        rec.species = int16_t(s);
        rec.wall = int16_t(wall);
        rec.cell = wcell;
        rec.step = *a.step;
        rec.vx = vx1;
        rec.vy = vy1;
        a.hits[h] = rec;
      } else {
        atomicOr(a.status, PIC_ST_FULL);
      }
      return 1;
    }
  }
  if (oi == cx && oj == cy) return 0;
  atomicOr(a.status, PIC_ST_CFL);   // moved farther than the walk limit: dropped untallied
  return 2;
}

// Ion recycling (Sec. III-A, III-C): the thermal ion that replaces an ion
// absorbed during step `step` keeps its id and enters at a uniform position
// of the source rows with a Maxwellian velocity, taken as its v^{n+1/2}.
// Draws: Philox4x32-10 with key = seed and counter (id, step, tag, k);
// k = 0 gives the cell (row, column by multiply-high) and the two in-cell
// offsets (top 24 bits, exact in FP32), k = 1 the Box-Muller pair.
__device__ __forceinline__ void recycled_ion(const PArgs &a, uint32_t id, int step, int &c, float &fx,
                                             float &fy, float &vx, float &vy) {
  const uint4 r = philox4x32_10(make_uint4(id, uint32_t(step), kTagRecycle, 0u), a.key);
  const uint4 q = philox4x32_10(make_uint4(id, uint32_t(step), kTagRecycle, 1u), a.key);
  const int i = a.src_x0 + int(below(r.x, uint32_t(a.src_rows)));
  const int j = int(below(r.y, uint32_t(a.g.ny)));
  c = pack_cell(i, j);
  fx = unit24(r.z);
  fy = unit24(r.w);
  const float rad = sqrtf(-2.0f * logf(unit24_open(q.x)));
  float sn, cs;
  sincospif(2.0f * unit24(q.y), &sn, &cs);
  vx = a.vth_i * (rad * cs);
  vy = a.vth_i * (rad * sn);
}

template <int MODE, int V>
__device__ __forceinline__ void move_one(const PArgs &a, const float2 *sE, uint32_t *sAcc,
                                         unsigned long long *acc, int s, int wi0, int wj0,
                                         const uint32_t *id, int64_t slot, int &c, float &fx,
                                         float &fy, float &vx, float &vy, float &ke) {
  if (c < 0) return;
  constexpr int WXc = Win<V>::WXc, WYc = Win<V>::WYc, NWY = Win<V>::NWY;
  const Geom &g = a.g;
  const int i = cell_i(c);
  const int j = cell_j(c);
  int li = i - wi0, lj = j - wj0;
  bool inw = (unsigned)li < (unsigned)WXc && (unsigned)lj < (unsigned)WYc;
  if (!inw && (g.px | g.py)) {   // the window may reach across a periodic edge
    li = local_coord(i, wi0, g.nx, g.px);
    lj = local_coord(j, wj0, g.ny, g.py);
    inw = (unsigned)li < (unsigned)WXc && (unsigned)lj < (unsigned)WYc;
  }
  if (MODE == 1) {
    // deposit only, at the current position
    int w00, w01, w10, w11;
    cic_weights(fx, fy, w00, w01, w10, w11);
    if (inw) deposit_shared<NWY>(sAcc, li, lj, w00, w01, w10, w11);
    else deposit_global(a, acc, i, j, w00, w01, w10, w11);
    return;
  }
  float2 e00, e01, e10, e11;
  if (inw) {
    const int k = li * NWY + lj;
    e00 = sE[k];
    e01 = sE[k + 1];
    e10 = sE[k + NWY];
    e11 = sE[k + NWY + 1];
  } else {
    int i1 = i + 1, j1 = j + 1;
    if (g.px && i1 == g.nxn) i1 = 0;
    if (g.py && j1 == g.nyn) j1 = 0;
    e00 = __ldg(&a.E[i * g.nyn + j]);
    e01 = __ldg(&a.E[i * g.nyn + j1]);
    e10 = __ldg(&a.E[i1 * g.nyn + j]);
    e11 = __ldg(&a.E[i1 * g.nyn + j1]);
  }
  const float gx = __fsub_rn(1.0f, fx), gy = __fsub_rn(1.0f, fy);
  const float ex = bilerp(fx, fy, gx, gy, e00.x, e01.x, e10.x, e11.x);
  const float ey = bilerp(fx, fy, gx, gy, e00.y, e01.y, e10.y, e11.y);
  if (MODE == 2) {
    if (a.kick[s]) {
      vx = __fmaf_rn(a.qdt[s], ex, vx);
      vy = __fmaf_rn(a.qdt[s], ey, vy);
    }
    return;
  }
  const float vx1 = __fmaf_rn(a.qdt[s], ex, vx);
  const float vy1 = __fmaf_rn(a.qdt[s], ey, vy);
  ke = __fadd_rn(ke, __fmaf_rn(vx, vx1, __fmul_rn(vy, vy1)));
  vx = vx1;
  vy = vy1;
  const float dx = __fmul_rn(vx1, a.dt), dy = __fmul_rn(vy1, a.dt);
  float nfx = __fadd_rn(fx, dx), nfy = __fadd_rn(fy, dy);
  const float cxf = floorf(nfx), cyf = floorf(nfy);
  const int cx = int(cxf), cy = int(cyf);
  int oi = 0, oj = 0;     // cell offset of the move
  if (cx | cy) {
    const bool near = (unsigned)(cx + 1) <= 2u && (unsigned)(cy + 1) <= 2u;
    if (near && (__ldg(&a.cellmask[i * g.ny + j]) & kCellInterior)) {
      // all eight neighbours are plasma: no face within one cell can absorb
      oi = cx;
      oj = cy;
    } else if (const int gone = walk_move(a, s, i, j, fx, fy, dx, dy, cx, cy, vx1, vy1, id, slot, oi, oj)) {
      if (gone == 1 && s == 1 && a.recycle) {
        // tallied above; a thermal ion takes its place and joins the deposit
        recycled_ion(a, id[slot], *a.step, c, fx, fy, vx, vy);
        int w00, w01, w10, w11;
        cic_weights(fx, fy, w00, w01, w10, w11);
        deposit_global(a, acc, cell_i(c), cell_j(c), w00, w01, w10, w11);
        return;
      }
      c = -1;   // absorbed and tallied, or moved beyond the walk limit
      return;
    }
    nfx = __fsub_rn(nfx, cxf);
    nfy = __fsub_rn(nfy, cyf);
    nfx = fminf(nfx, 0x1.fffffep-1f);
    nfy = fminf(nfy, 0x1.fffffep-1f);
    int ni = i + oi, nj = j + oj;
    if (g.px) ni = wrapmod(ni, g.nx);
    if (g.py) nj = wrapmod(nj, g.ny);
    c = pack_cell(ni, nj);
  }
  fx = nfx;
  fy = nfy;
  // deposit at the new position; window coordinates follow the move unwrapped
  int w00, w01, w10, w11;
  cic_weights(fx, fy, w00, w01, w10, w11);
  const int lni = li + oi, lnj = lj + oj;
  if ((unsigned)lni < (unsigned)WXc && (unsigned)lnj < (unsigned)WYc) {
    deposit_shared<NWY>(sAcc, lni, lnj, w00, w01, w10, w11);
  } else {
    deposit_global(a, acc, cell_i(c), cell_j(c), w00, w01, w10, w11);
  }
}

// The step kernel asks for the particle state of its next iteration (512
// particles, one bulk L2 prefetch per array from thread 0) while the CTA
// works on the current one, so the next loads find it in L2.  One iteration
// ahead measured best (further ahead, or on into the next chunk, was slower).
constexpr int kPrefetchAhead = 1;
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int MODE, int V>
__global__ void __launch_bounds__(Win<V>::THREADS, 1024 / Win<V>::THREADS) k_particles(PArgs a) {
  constexpr int NWX = Win<V>::NWX, NWY = Win<V>::NWY, THREADS = Win<V>::THREADS;
  __shared__ float2 sE[NWX * NWY];
  __shared__ uint32_t sAcc[NWX * NWY];
  __shared__ double sRed[THREADS / 32];
  const Geom g = a.g;
  const int nch = *a.nchunks;
  const int nnodes = g.nxn * g.nyn;
  if (MODE == 0 && blockIdx.x == 0 && threadIdx.x == 0) a.fe[1] = a.fe[0];
  for (int ci = blockIdx.x; ci < nch; ci += gridDim.x) {
    const Chunk ch = a.chunks[ci];
    const int s = ch.species;
    const int ti = ch.tile / g.nty;
    const int tj = ch.tile - ti * g.nty;
    const int wi0 = ti * Win<V>::TX - Win<V>::H;
    const int wj0 = tj * Win<V>::TY - Win<V>::H;
    for (int k = threadIdx.x; k < NWX * NWY; k += blockDim.x) {
      if (MODE != 1) {
        const int wi = k / NWY, wj = k - (k / NWY) * NWY;
        int gi = wi0 + wi, gj = wj0 + wj;
        if (g.px) gi = wrapmod(gi, g.nxn);
        if (g.py) gj = wrapmod(gj, g.nyn);
        float2 e = make_float2(0.f, 0.f);
        if (gi >= 0 && gi < g.nxn && gj >= 0 && gj < g.nyn) e = a.E[gi * g.nyn + gj];
        sE[k] = e;
      }
      sAcc[k] = 0u;
    }
    __syncthreads();
    unsigned long long *acc = a.acc + (int64_t)s * nnodes;
    const ParticleBuf P = a.pbufs[2 * s + a.cur[s]];
    float ke = 0.f;
    // L2 prefetch of the particle state kPrefetchAhead iterations ahead
    const int64_t step = 4 * int64_t(blockDim.x);
    auto prefetch = [&](int64_t from) {
      if (MODE == 0 && threadIdx.x == 0 && from < ch.end) {
        const unsigned bytes = unsigned(min((long long)step, (long long)ch.end - from)) * 4u;
        prefetch_l2(P.cell + from, bytes);
        prefetch_l2(P.fx + from, bytes);
        prefetch_l2(P.fy + from, bytes);
        prefetch_l2(P.vx + from, bytes);
        prefetch_l2(P.vy + from, bytes);
      }
    };
    for (int d = 0; d < kPrefetchAhead; ++d) prefetch(int64_t(ch.begin) + d * step);
    for (int64_t base = ch.begin + 4 * threadIdx.x; base < ch.end; base += 4 * blockDim.x) {
      prefetch(base - 4 * threadIdx.x + kPrefetchAhead * step);
      int4 c4 = *reinterpret_cast<const int4 *>(P.cell + base);
      float4 fx4 = *reinterpret_cast<const float4 *>(P.fx + base);
      float4 fy4 = *reinterpret_cast<const float4 *>(P.fy + base);
      float4 vx4 = make_float4(0.f, 0.f, 0.f, 0.f), vy4 = vx4;
      if (MODE != 1) {
        vx4 = *reinterpret_cast<const float4 *>(P.vx + base);
        vy4 = *reinterpret_cast<const float4 *>(P.vy + base);
      }
      move_one<MODE, V>(a, sE, sAcc, acc, s, wi0, wj0, P.id, base + 0, c4.x, fx4.x, fy4.x, vx4.x, vy4.x, ke);
      move_one<MODE, V>(a, sE, sAcc, acc, s, wi0, wj0, P.id, base + 1, c4.y, fx4.y, fy4.y, vx4.y, vy4.y, ke);
      move_one<MODE, V>(a, sE, sAcc, acc, s, wi0, wj0, P.id, base + 2, c4.z, fx4.z, fy4.z, vx4.z, vy4.z, ke);
      move_one<MODE, V>(a, sE, sAcc, acc, s, wi0, wj0, P.id, base + 3, c4.w, fx4.w, fy4.w, vx4.w, vy4.w, ke);
      if (MODE == 0) {   // streaming stores: the written state is not read again this step
        __stcs(reinterpret_cast<int4 *>(P.cell + base), c4);
        __stcs(reinterpret_cast<float4 *>(P.fx + base), fx4);
        __stcs(reinterpret_cast<float4 *>(P.fy + base), fy4);
        __stcs(reinterpret_cast<float4 *>(P.vx + base), vx4);
        __stcs(reinterpret_cast<float4 *>(P.vy + base), vy4);
      } else if (MODE != 1) {
        *reinterpret_cast<float4 *>(P.vx + base) = vx4;
        *reinterpret_cast<float4 *>(P.vy + base) = vy4;
      }
    }
    __syncthreads();
    if (MODE != 2) {
      for (int k = threadIdx.x; k < NWX * NWY; k += blockDim.x) {
        const uint32_t v = sAcc[k];
        if (v) {
          const int wi = k / NWY, wj = k - (k / NWY) * NWY;
          int gi = wi0 + wi, gj = wj0 + wj;
          if (g.px) gi = wrapmod(gi, g.nxn);
          if (g.py) gj = wrapmod(gj, g.nyn);
          // The node's sum over the chunk lies in [-kChunk, kChunk * 2^20]: each of
          // at most kChunk particles adds a share in [-1, 2^20].  That range is
          // narrower than 2^32, so the 32-bit sum decodes uniquely; values above
          // kChunk * 2^20 are the negative ones.
          const long long x = v > uint32_t(kChunk) * kQ ? (long long)v - (1ll << 32) : (long long)v;
          if (gi >= 0 && gi < g.nxn && gj >= 0 && gj < g.nyn)
            atomicAdd(&acc[gi * g.nyn + gj], (unsigned long long)x);
        }
      }
    }
    if (MODE == 0) {
      float v = ke;   // FP32 within the warp, FP64 from the warps' sums on
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) sRed[threadIdx.x >> 5] = double(v);
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) t += sRed[w];
        a.ke_part[ci] = t;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Load conversion, export, reductions
// ---------------------------------------------------------------------------
__global__ void k_load_convert(ParticleBuf P, Geom g, const uint8_t *cellmask, const double *x,
                               const double *y, const double *vx, const double *vy,
                               const uint32_t *id, int64_t offset, int64_t n, uint32_t *status) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double X = x[k], Y = y[k];
  // (the reduction into a periodic box only for coordinates outside it: FP64
  // remainders are long instruction sequences here)
  if (g.px && !(X >= 0.0 && X < double(g.nx))) {
    X = fmod(X, double(g.nx));
    if (X < 0) X += g.nx;
    if (X >= g.nx) X -= g.nx;
  }
  if (g.py && !(Y >= 0.0 && Y < double(g.ny))) {
    Y = fmod(Y, double(g.ny));
    if (Y < 0) Y += g.ny;
    if (Y >= g.ny) Y -= g.ny;
  }
  const double fi = floor(X), fj = floor(Y);
  int c = -1;
  float fx = 0.f, fy = 0.f;
  if (X == X && Y == Y && fi >= 0 && fi < g.nx && fj >= 0 && fj < g.ny) {
    const int i = int(fi), j = int(fj);
    if (cellmask[i * g.ny + j]) {
      c = (i << 16) | j;
      fx = fminf(float(X - fi), 0x1.fffffep-1f);
      fy = fminf(float(Y - fj), 0x1.fffffep-1f);
    }
  }
  if (c < 0) atomicOr(status, PIC_ST_RANGE);
  const int64_t d = offset + k;
  P.cell[d] = c;
  P.fx[d] = fx;
  P.fy[d] = fy;
  P.vx[d] = float(vx[k]);
  P.vy[d] = float(vy[k]);
  P.id[d] = id ? id[k] : uint32_t(offset + k);
}

__global__ void k_export(ParticleBuf P, Geom g, const int64_t *nslots_p, double *out, int64_t cap,
                         unsigned long long *counter) {
  const int64_t nslots = *nslots_p;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < nslots; base += nwarps * 32) {
    const int64_t p = base + lane;
    const int c = p < nslots ? P.cell[p] : -1;
    const unsigned live = __ballot_sync(0xffffffffu, c >= 0);
    unsigned long long b = 0;
    if (lane == 0 && live) b = atomicAdd(counter, (unsigned long long)__popc(live));
    b = __shfl_sync(0xffffffffu, b, 0);
    if (c >= 0) {
      const int64_t d = int64_t(b) + __popc(live & ((1u << lane) - 1u));
      if (d < cap) {
        const int i = cell_i(c), j = cell_j(c);
        out[d] = double(i) + double(P.fx[p]);
        out[cap + d] = double(j) + double(P.fy[p]);
        out[2 * cap + d] = double(P.vx[p]);
        out[3 * cap + d] = double(P.vy[p]);
        out[4 * cap + d] = double(P.id[p]);
      }
    }
  }
}

// Live particles of one species in their stored form (cell, offsets,
// velocities, id), compacted into out (a checkpoint); order arbitrary.
__global__ void k_export_raw(ParticleBuf P, const int64_t *nslots_p, ParticleBuf out, int64_t cap,
                             unsigned long long *counter) {
  const int64_t nslots = *nslots_p;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < nslots; base += nwarps * 32) {
    const int64_t p = base + lane;
    const int c = p < nslots ? P.cell[p] : -1;
    const unsigned live = __ballot_sync(0xffffffffu, c >= 0);
    unsigned long long b = 0;
    if (lane == 0 && live) b = atomicAdd(counter, (unsigned long long)__popc(live));
    b = __shfl_sync(0xffffffffu, b, 0);
    if (c >= 0) {
      const int64_t d = int64_t(b) + __popc(live & ((1u << lane) - 1u));
      if (d < cap) {
        out.cell[d] = c;
        out.fx[d] = P.fx[p];
        out.fy[d] = P.fy[p];
        out.vx[d] = P.vx[p];
        out.vy[d] = P.vy[p];
        out.id[d] = P.id[p];
      }
    }
  }
}

// per-block partial sums of [vx, vy, live] of one species
__global__ void k_moments(ParticleBuf P, const int64_t *nslots_p, double *part) {
  const int64_t nslots = *nslots_p;
  double sx = 0, sy = 0, sn = 0;
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < nslots;
       p += int64_t(gridDim.x) * blockDim.x) {
    if (P.cell[p] >= 0) {
      sx += P.vx[p];
      sy += P.vy[p];
      sn += 1.0;
    }
  }
  __shared__ double r[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_down_sync(0xffffffffu, sx, o);
    sy += __shfl_down_sync(0xffffffffu, sy, o);
    sn += __shfl_down_sync(0xffffffffu, sn, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    r[0][w] = sx;
    r[1][w] = sy;
    r[2][w] = sn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, n = 0;
    for (int k = 0; k < int(blockDim.x >> 5); ++k) {
      a += r[0][k];
      b += r[1][k];
      n += r[2][k];
    }
    part[3 * blockIdx.x + 0] = a;
    part[3 * blockIdx.x + 1] = b;
    part[3 * blockIdx.x + 2] = n;
  }
}

template <int MODE, int V>
cudaError_t launch_particles_v(pic_ctx *c, const PArgs &a) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_particles<0, V>, Win<V>::THREADS, 0);
  if (per_sm < 1) per_sm = 1;
  k_particles<MODE, V><<<c->num_sms * per_sm, Win<V>::THREADS, 0, c->stream>>>(a);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_particles_mode(pic_ctx *c, const PArgs &a) {
  switch (c->tile_variant) {
    case 1: return launch_particles_v<MODE, 1>(c, a);
    case 2: return launch_particles_v<MODE, 2>(c, a);
    case 3: return launch_particles_v<MODE, 3>(c, a);
    default: return launch_particles_v<MODE, 0>(c, a);
  }
}

}  // namespace

cudaError_t launch_sort(pic_ctx *c) {
  SortArgs a;
  a.pbufs = c->d_pbufs;
  a.cur = c->d_cur;
  a.nslots = c->d_nslots;
  a.count = c->d_tile_count;
  a.cursor = c->d_tile_cursor;
  a.start = c->d_tile_start;
  a.chunks = c->d_chunks;
  a.nchunks = c->d_nchunks;
  a.nslots_out = c->d_nslots + 2;
  a.g = c->g;
  a.ntiles = c->g.ntx * c->g.nty;
  const dim3 grid(c->num_sms * 8, 2);   // 8 CTAs of 256 threads per SM and species
  if (a.ntiles <= kHistSmemTiles)
    k_sort_hist<true><<<grid, 256, size_t(a.ntiles) * 4, c->stream>>>(a);
  else
    k_sort_hist<false><<<grid, 256, 0, c->stream>>>(a);
  k_sort_scan<<<1, 1024, 0, c->stream>>>(a);
  k_sort_scatter<<<grid, 256, 0, c->stream>>>(a);
  k_sort_finish<<<1, 1, 0, c->stream>>>(c->d_nslots, c->d_cur);
  for (int s = 0; s < 2; ++s) c->cur[s] ^= 1;
  return cudaGetLastError();
}

cudaError_t launch_particles(pic_ctx *c, int mode, float kick_factor, const int *species_mask) {
  PArgs a;
  a.pbufs = c->d_pbufs;
  a.cur = c->d_cur;
  for (int s = 0; s < 2; ++s) {
    a.qdt[s] = float(c->cfg.alpha[s] * c->cfg.dt * kick_factor);
    a.kick[s] = species_mask ? species_mask[s] : 1;
  }
  a.chunks = c->d_chunks;
  a.nchunks = c->d_nchunks;
  a.E = c->d_E;
  a.acc = c->d_acc;
  a.cellmask = c->d_cellmask;
  a.g = c->g;
  a.dt = float(c->cfg.dt);
  a.walls = c->d_walls;
  a.bottom = c->d_bottom;
  a.hits = c->d_hits;
  a.nhits = c->d_nhits;
  a.hit_cap = c->cfg.hit_capacity;
  a.status = c->d_status;
  a.step = c->d_step;
  a.ke_part = c->d_ke_part;
  a.fe = c->d_fe;
  a.recycle = c->cfg.recycle ? 1 : 0;
  a.src_x0 = c->src_x0;
  a.src_rows = c->src_x1 - c->src_x0;
  a.key = make_uint2(uint32_t(c->cfg.seed), uint32_t(c->cfg.seed >> 32));
  a.vth_i = float(c->cfg.recycle_vth);
  switch (mode) {
    case 0: return launch_particles_mode<0>(c, a);
    case 1: return launch_particles_mode<1>(c, a);
    default: return launch_particles_mode<2>(c, a);
  }
}

void set_tile_variant(pic_ctx *c, int v) {
  const TileVariant &t = kTileVariants[v];
  c->tile_variant = v;
  c->g.tsx = t.log2x;
  c->g.tsy = t.log2y;
  c->g.ntx = (c->g.nx + (1 << t.log2x) - 1) >> t.log2x;
  c->g.nty = (c->g.ny + (1 << t.log2y) - 1) >> t.log2y;
  c->needs_sort = 1;
}

cudaError_t launch_load_convert(pic_ctx *c, int s, const double *d_x, const double *d_y,
                                const double *d_vx, const double *d_vy, const uint32_t *d_id,
                                int64_t offset, int64_t n) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_load_convert<<<dim3((unsigned)blocks), 256, 0, c->stream>>>(
      c->pb[s][c->cur[s]], c->g, c->d_cellmask, d_x, d_y, d_vx, d_vy, d_id, offset, n,
      c->d_status);
  return cudaGetLastError();
}

cudaError_t launch_export_state(pic_ctx *c, int s, double *d_out, int64_t cap,
                                unsigned long long *d_counter) {
  k_export<<<c->num_sms * 4, 256, 0, c->stream>>>(c->pb[s][c->cur[s]], c->g, c->d_nslots + s,
                                                   d_out, cap, d_counter);
  return cudaGetLastError();
}

cudaError_t launch_export_raw(pic_ctx *c, int s, ParticleBuf out, int64_t cap,
                              unsigned long long *d_counter) {
  k_export_raw<<<c->num_sms * 4, 256, 0, c->stream>>>(c->pb[s][c->cur[s]], c->d_nslots + s, out, cap,
                                                       d_counter);
  return cudaGetLastError();
}

cudaError_t launch_moments(pic_ctx *c, int s, double *d_part, int nblocks) {
  k_moments<<<nblocks, 256, 0, c->stream>>>(c->pb[s][c->cur[s]], c->d_nslots + s, d_part);
  return cudaGetLastError();
}

}  // namespace picgb
