// binning.cu -- tile-key duplication and sorting of (Gaussian, tile)
// instances, per frame of a batch.
//
// The instance order is that of a stable sort of the 64-bit keys
// (frame * tiles + tile) << 32 | bits(z), with instances emitted in Gaussian
// order (so equal keys stay in index order).  It is computed as an LSD radix
// sort whose low digits (the 32 depth bits) are applied to the Gaussians
// BEFORE duplication -- they are a per-Gaussian key -- and whose high digit
// (frame, tile) is one stable counting pass over the duplicated instances:
//   1. depth sort: 4 passes of 8 bits over the per-frame depth keys
//      (culled Gaussians carry 0xFFFFFFFF and are left out), each tile of
//      keys ranked in shared memory and written out in digit order; the last
//      pass also writes each Gaussian's tile rectangle and tile count in
//      depth order;
//   2. emission offsets: exclusive scan (one pass, decoupled look-back) of
//      the tiles each depth-ordered Gaussian covers, counted by the last
//      depth-sort pass; chunks of kChunk consecutive instances per frame;
//   3. per chunk, tile counts: every Gaussian (or the part of its rectangle
//      inside the chunk) adds +-1 at the corners of its tile rectangle in a
//      difference array, whose 2D prefix sum is the count of each tile
//      (also summed into per-tile totals); a scan over each frame's chunks
//      per tile, and over its tiles, gives the tile ranges;
//   4. scatter: per warp of a chunk the same corner counts give its cursors;
//      then the warp deals its instances out 32 at a time in emission order,
//      each lane writing its Gaussian's index at its tile's running cursor
//      (lanes of one tile in lane order: stable by construction).
// The 64-bit keys themselves are never needed by the compositing kernels;
// gftorf_export_tile_lists materialises them from the ranges.
#include "gftorf_internal.cuh"

namespace gftorf {
namespace {

// Exclusive scan in place of a[0..S) by one CTA; returns the total through
// *total (if non-null).  Each thread scans a contiguous segment.
template <typename T>
__device__ void cta_exclusive_scan(T* a, int64_t S, uint64_t* total) {
  __shared__ uint64_t s_warp[32];
  const int nt = blockDim.x, tid = threadIdx.x;
  const int64_t seg = (S + nt - 1) / nt;
  const int64_t lo = min((int64_t)tid * seg, S), hi = min(lo + seg, S);
  uint64_t sum = 0;
  for (int64_t i = lo; i < hi; ++i) sum += a[i];
  // block exclusive scan of the segment sums
  const int lane = tid & 31, wid = tid >> 5;
  uint64_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = (nt + 31) / 32;
    uint64_t v = lane < nw ? s_warp[lane] : 0;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < nw) s_warp[lane] = x - v;  // exclusive warp offsets
  }
  __syncthreads();
  uint64_t run = s_warp[wid] + incl - sum;
  for (int64_t i = lo; i < hi; ++i) {
    const uint64_t v = a[i];
    a[i] = (T)run;
    run += v;
  }
  if (total && tid == nt - 1) *total = run;
  __syncthreads();
}

// Largest r in [0, n) with e[r] <= s, for e strictly increasing and
// e[0] <= s; one 32-way probe per step by the calling warp.
__device__ __forceinline__ int warp_upper_rank(const uint32_t* __restrict__ e, int n,
                                               uint32_t s, int lane) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) / 32;
    const int probe = lo + lane * step;
    const bool ok = probe < hi && e[probe] <= s;
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    const int last = 31 - __clz(m);
    lo += last * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

// ---------------------------------------------------------------------------
// tile counts of rectangles from their corners
// ---------------------------------------------------------------------------
// A rectangle [xa, xb) x [ya, yb) of tiles adds +1 at (xa, ya) and (xb, yb)
// and -1 at (xb, ya) and (xa, yb) of a (tiles_y + 1) x (tiles_x + 1)
// difference array D (row stride `cols` = tiles_x + 1, arithmetic mod 2^32);
// the inclusive 2D prefix sum of D is then, at every tile, the number of
// rectangles covering it.
__device__ __forceinline__ void diff_add_rect(uint32_t* D, int cols, int xa, int ya, int xb,
                                              int yb) {
  if (xa >= xb || ya >= yb) return;
  atomicAdd(&D[ya * cols + xa], 1u);
  atomicAdd(&D[ya * cols + xb], 0xFFFFFFFFu);
  atomicAdd(&D[yb * cols + xa], 0xFFFFFFFFu);
  atomicAdd(&D[yb * cols + xb], 1u);
}

// The instances [lo, hi) (row-major indices, hi > lo) of a Gaussian whose
// tile rectangle is w x h and starts at (x0, y0): the whole rectangle (the
// usual case), else at most three rectangles (the tail of a first row, whole
// rows, the head of a last row).
__device__ __forceinline__ void diff_add_span(uint32_t* D, int cols, int x0, int y0, int w,
                                              int h, int lo, int hi) {
  if (lo == 0 && hi == w * h) {
    diff_add_rect(D, cols, x0, y0, x0 + w, y0 + h);
    return;
  }
  const int ky0 = lo / w, kx0 = lo - ky0 * w;
  const int last = hi - 1;
  const int ky1 = last / w, kx1 = last - ky1 * w;
  if (ky0 == ky1) {
    diff_add_rect(D, cols, x0 + kx0, y0 + ky0, x0 + kx1 + 1, y0 + ky0 + 1);
  } else if (kx0 == 0 && kx1 == w - 1) {
    diff_add_rect(D, cols, x0, y0 + ky0, x0 + w, y0 + ky1 + 1);
  } else {
    diff_add_rect(D, cols, x0 + kx0, y0 + ky0, x0 + w, y0 + ky0 + 1);
    diff_add_rect(D, cols, x0, y0 + ky0 + 1, x0 + w, y0 + ky1);
    diff_add_rect(D, cols, x0, y0 + ky1, x0 + kx1 + 1, y0 + ky1 + 1);
  }
}

// Corner counts of the depth-ordered Gaussians r0, r0 + stride, ... (below
// vis) whose instances meet [s, e): four Gaussians' offsets and rectangles
// loaded at once per step (emission offsets increase with r, so the first
// Gaussian starting at or past e ends the walk).
__device__ __forceinline__ void diff_add_gaussians(uint32_t* D, int cols,
                                                   const uint32_t* __restrict__ eb,
                                                   const uint2* __restrict__ rc, int r0,
                                                   int stride, int vis, uint32_t s, uint32_t e) {
  constexpr int U = 4;
  for (int r = r0; r < vis; r += U * stride) {
    uint32_t eo[U];
    uint2 rr[U];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const int ri = r + i * stride;
      eo[i] = ri < vis ? eb[ri] : 0xFFFFFFFFu;
      rr[i] = ri < vis ? rc[ri] : make_uint2(0u, 0u);
    }
    bool stop = false;
#pragma unroll
    for (int i = 0; i < U; ++i) {
      if (stop || eo[i] >= e) {
        stop = true;
      } else {
        int x0, y0, x1, y1;
        unpack_rect(rr[i], x0, y0, x1, y1);
        const int w = x1 - x0;
        const uint32_t n = (uint32_t)(w * (y1 - y0));
        const uint32_t lo = max(s, eo[i]) - eo[i], hi = min(e, eo[i] + n) - eo[i];
        diff_add_span(D, cols, x0, y0, w, y1 - y0, (int)lo, (int)hi);
      }
    }
    if (stop) break;
  }
}

// Inclusive 2D prefix sum of D (rows x cols) by threads [0, nthr) of a group
// (a warp: WARP = true, else the whole CTA): a sequential scan per row, then
// per column.
template <bool WARP>
__device__ __forceinline__ void prefix2d(uint32_t* D, int rows, int cols, int tid, int nthr) {
  for (int y = tid; y < rows; y += nthr) {
    uint32_t* row = D + y * cols;
    uint32_t run = 0;
    for (int x = 0; x < cols; ++x) {
      run += row[x];
      row[x] = run;
    }
  }
  if (WARP)
    __syncwarp();
  else
    __syncthreads();
  for (int x = tid; x < cols; x += nthr) {
    uint32_t run = 0;
    for (int y = 0; y < rows; ++y) {
      run += D[y * cols + x];
      D[y * cols + x] = run;
    }
  }
}

// ---------------------------------------------------------------------------
// footprints given by the caller (binning-only entry point)
// ---------------------------------------------------------------------------
__global__ void footprint_kernel(const float* __restrict__ u,
                                 const float* __restrict__ v,
                                 const int32_t* __restrict__ radius,
                                 const float* __restrict__ z,
                                 Header* __restrict__ hdr,
                                 uint2* __restrict__ rect,
                                 uint32_t* __restrict__ zkey, int N, int TW,
                                 int TH, int tiles_x, int tiles_y) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  bool visible = false;
  if (g < N) {
    const size_t i = (size_t)b * N + g;
    uint2 rr = make_uint2(0, 0);
    uint32_t key = kCulledKey;
    const int r = radius[i];
    if (r > 0) {
      int x0, y0, x1, y1;
      tile_rect(u[i], v[i], r, TW, TH, tiles_x, tiles_y, x0, y0, x1, y1);
      if (x0 < x1 && y0 < y1) {
        visible = true;
        rr = pack_rect(x0, y0, x1, y1);
        key = __float_as_uint(z[i]);
      }
    }
    rect[i] = rr;
    zkey[i] = key;
  }
  const unsigned m = __ballot_sync(0xffffffffu, visible);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(&hdr->vis[b], (uint32_t)__popc(m));
}

// ---------------------------------------------------------------------------
// depth sort: stable LSD radix sort, 8-bit digits, one segment per frame.
// The per-frame digit totals of all four passes come from one reading of the
// keys (they do not depend on the order); each pass is then one kernel that
// ranks a tile of keys in shared memory and finds the tile's offset for each
// digit from the tiles before it (decoupled look-back: every tile publishes
// its digit counts, then the running prefix once it knows it).  Culled
// Gaussians (key 0xFFFFFFFF) are left out: their place in the order is never
// read (every later kernel stops at the frame's visible count), so the first
// pass packs the visible keys at the front of the frame and the later passes
// run only the frame's ceil(visible / 2048) tiles.
// ---------------------------------------------------------------------------
constexpr uint32_t kLbPrefix = 0x80000000u;  // status word: inclusive prefix
constexpr uint32_t kLbAggregate = 0x40000000u;  // status word: this tile's count only
constexpr uint32_t kLbCount = 0x3FFFFFFFu;
constexpr int kLbSpinLimit = 1 << 22;  // bounded wait on a predecessor tile

__global__ void __launch_bounds__(kSortThreads)
    dsort_hist_kernel(const uint32_t* __restrict__ keys, int N, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[4][256];
  const int blk = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
  for (int i = tid; i < 4 * 256; i += kSortThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const uint32_t* k = keys + (size_t)b * N;
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const int pos = blk * kSortTile + it * kSortThreads + tid;
    if (pos < N) {
      const uint32_t key = k[pos];
      if (key != kCulledKey) {
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&h[p][(key >> (8 * p)) & 255u], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < 4 * 256; i += kSortThreads) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&ghist[(size_t)b * 1024 + i], c);
  }
}

// per (frame, pass): exclusive scan of the 256 digit totals -> digit bases.
// The same CTAs clear the later stages' per-step words: the per-(frame,
// tile) instance totals and the emission scan's status words and counters.
__global__ void __launch_bounds__(256)
    dsort_bases_kernel(uint32_t* __restrict__ ghist, uint32_t* __restrict__ ttot, int n_ttot,
                       uint64_t* __restrict__ scan_state, int n_state) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_ttot; i += gridDim.x * blockDim.x)
    ttot[i] = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_state; i += gridDim.x * blockDim.x)
    scan_state[i] = 0;
  cta_exclusive_scan<uint32_t>(ghist + (size_t)blockIdx.x * 256, 256, nullptr);
}

// One pass: tiles are claimed in order through an atomic counter, so a tile
// only ever waits for tiles that are already running.  rin/rout (last pass
// only, else null): the Gaussians' tile rectangles are written in the
// sorted order as well.
__global__ void __launch_bounds__(kSortThreads, 5)  // <= 48 registers, no spill
    dsort_pass_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ iin,
                      uint32_t* __restrict__ kout, uint32_t* __restrict__ iout, int N, int B,
                      int pass, int n_dblk, const uint32_t* __restrict__ gbase,
                      uint32_t* __restrict__ status, uint32_t* __restrict__ tile_counter,
                      Header* __restrict__ hdr, const uint2* __restrict__ rin,
                      uint2* __restrict__ rout, uint32_t* __restrict__ ecnt) {
  __shared__ uint32_t wc[kSortWarps][256];
  __shared__ uint32_t s_tile;
  // the tile's keys and indices in digit order (staged, then written out in
  // runs of consecutive places), each digit's first place in the tile and in
  // the frame, the warps' digit-count sums
  __shared__ uint32_t s_key[kSortTile], s_id[kSortTile];
  __shared__ uint32_t s_tstart[256], s_gbase[256], s_wsum[kSortWarps];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int shift = 8 * pass;
  if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
  for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&wc[0][0])[i] = 0;
  __syncthreads();
  const uint32_t L = s_tile;
  const int b = (int)(L / (uint32_t)n_dblk), blk = (int)(L - (uint32_t)b * n_dblk);
  const size_t fb = (size_t)b * N;
  const int start = blk * kSortTile + w * (kSortTile / kSortWarps);
  // the first pass reads all N keys of the frame (culled ones skipped), the
  // later ones the visible keys packed at its front
  const int vis = (int)hdr->vis[b];
  const int n_in = pass == 0 ? N : vis;
  if (ecnt) {  // last pass: the tile's places past the visible count cover no tiles
    const int z0 = max(vis, blk * kSortTile), z1 = min(N, (blk + 1) * kSortTile);
    for (int p = z0 + tid; p < z1; p += kSortThreads) ecnt[fb + p] = 0u;
  }
  if (blk * kSortTile >= n_in) return;  // no keys: no later tile waits for it
  uint32_t key[kSortItems], id[kSortItems], loc[kSortItems];
  bool live[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {  // all loads in flight first
    const int pos = start + it * 32 + lane;
    const bool valid = pos < n_in;
    key[it] = valid ? kin[fb + pos] : kCulledKey;
    id[it] = valid ? (iin ? iin[fb + pos] : (uint32_t)pos) : 0u;
  }
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) live[it] = key[it] != kCulledKey;
  // rank within the warp (lanes in order, items in order): stable.  The
  // lanes sharing a digit in each item first (independent of one another:
  // eight ballots, one per digit bit, measured faster than match.any), then
  // the warp's running digit counts item after item.
  uint32_t peers[kSortItems];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    // lanes with the same digit: one ballot per digit bit (live lanes only)
    const uint32_t d = (key[it] >> shift) & 255u;
    unsigned pm = __ballot_sync(0xffffffffu, live[it]);
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
      const bool on = (d >> bit) & 1u;
      const unsigned bm = __ballot_sync(0xffffffffu, on);
      pm &= on ? bm : ~bm;
    }
    peers[it] = live[it] ? pm : (1u << lane);
  }
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const bool valid = live[it];
    const uint32_t d = (key[it] >> shift) & 255u;
    const uint32_t rank = __popc(peers[it] & lt);
    const uint32_t before = valid ? wc[w][d] : 0u;
    __syncwarp();
    if (valid && rank == 0) wc[w][d] = before + __popc(peers[it]);
    __syncwarp();
    loc[it] = before + rank;
  }
  __syncthreads();
  {
    const int d = tid;  // 256 threads, one digit each
    uint32_t cnt = 0;
#pragma unroll
    for (int ww = 0; ww < kSortWarps; ++ww) {
      const uint32_t t = wc[ww][d];
      wc[ww][d] = cnt;
      cnt += t;
    }
    // publish this tile's count, then find the count of the tiles before it
    volatile uint32_t* st = status + ((size_t)pass * B + b) * (size_t)n_dblk * 256;
    uint32_t excl = 0;
    if (blk == 0) {
      st[d] = kLbPrefix | cnt;
    } else {
      st[(size_t)blk * 256 + d] = kLbAggregate | cnt;
      int j = blk - 1, spins = 0;
      for (;;) {
        const uint32_t v = st[(size_t)j * 256 + d];
        if (v == 0u) {
          if (++spins > kLbSpinLimit) {  // never expected: tiles before are running
            set_status(hdr, GFTORF_ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
          continue;
        }
        excl += v & kLbCount;
        if ((v & kLbPrefix) || j == 0) break;
        --j;
      }
      st[(size_t)blk * 256 + d] = kLbPrefix | (excl + cnt);
    }
    s_gbase[d] = gbase[((size_t)b * 4 + pass) * 256 + d] + excl;
    // first place of digit d in the tile: exclusive scan of the counts
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_wsum[w] = incl;
    __syncthreads();
    uint32_t before = 0;
#pragma unroll
    for (int ww = 0; ww < kSortWarps; ++ww) before += ww < w ? s_wsum[ww] : 0u;
    s_tstart[d] = before + incl - cnt;
  }
  __syncthreads();
  // stage in digit order: place = digit start + earlier warps' count of the
  // digit + rank in the warp
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    if (live[it]) {
      const uint32_t d = (key[it] >> shift) & 255u;
      const uint32_t tp = s_tstart[d] + wc[w][d] + loc[it];
      s_key[tp] = key[it];
      s_id[tp] = id[it];
    }
  }
  __syncthreads();
  // write out: consecutive threads take consecutive staged places, which lie
  // in runs of one digit at consecutive places of the frame
  uint32_t n_live = 0;
#pragma unroll
  for (int ww = 0; ww < kSortWarps; ++ww) n_live += s_wsum[ww];
  if (!rout) {
    for (uint32_t p = tid; p < n_live; p += kSortThreads) {
      const uint32_t k = s_key[p], g = s_id[p];
      const uint32_t d = (k >> shift) & 255u;
      const uint32_t dst = s_gbase[d] + (p - s_tstart[d]);
      if (dst < (uint32_t)vis) {  // always (a timed-out wait leaves garbage, not a fault)
        kout[fb + dst] = k;
        iout[fb + dst] = g;
      }
    }
    return;
  }
  // last pass: indices, rectangles and tile counts in depth order (the keys
  // are not needed again); the rectangles' gathers of four places at once
  constexpr int G = 4;
#pragma unroll 1
  for (uint32_t p0 = tid; p0 < n_live; p0 += G * kSortThreads) {
    uint32_t gg[G], dd[G];
    uint2 rr[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const uint32_t p = p0 + i * kSortThreads;
      dd[i] = 0xFFFFFFFFu;
      gg[i] = 0u;
      rr[i] = make_uint2(0u, 0u);
      if (p < n_live) {
        const uint32_t k = s_key[p], g = s_id[p];
        const uint32_t d = (k >> shift) & 255u;
        const uint32_t dst = s_gbase[d] + (p - s_tstart[d]);
        if (dst < (uint32_t)vis) {  // always (a timed-out wait leaves garbage, not a fault)
          dd[i] = dst;
          gg[i] = g;
          rr[i] = rin[fb + g];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < G; ++i) {
      if (dd[i] != 0xFFFFFFFFu) {
        iout[fb + dd[i]] = gg[i];
        rout[fb + dd[i]] = rr[i];
        int x0, y0, x1, y1;
        unpack_rect(rr[i], x0, y0, x1, y1);
        ecnt[fb + dd[i]] = (uint32_t)((x1 - x0) * (y1 - y0));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// emission offsets: tiles covered by each depth-ordered Gaussian (written by
// the last depth-sort pass), scanned over the whole batch (frame-major), so
// instance k of the batch is tile (k - e[g]) of Gaussian g's rectangle
// (row-major) for the g with e[g] <= k < e[g + 1].  One pass: tiles of
// kScanTile counts claimed in order through an atomic counter, each finding
// the sum of the tiles before it by decoupled look-back on 64-bit status
// words; the CTA that finishes last writes the chunk table (first instance
// and first binning chunk of each frame; chunks never straddle frames).
// ---------------------------------------------------------------------------
constexpr uint64_t kScanPrefix = 1ull << 63;     // status word: inclusive prefix
constexpr uint64_t kScanAggregate = 1ull << 62;  // status word: this tile's sum only
constexpr uint64_t kScanValue = kScanAggregate - 1;

__global__ void __launch_bounds__(kScanThreads)
    emission_scan_kernel(uint32_t* __restrict__ a, int64_t S, uint64_t* __restrict__ state,
                         int nblk, Header* __restrict__ hdr, int B, int N, int64_t cap,
                         int n_chunk) {
  constexpr int kItems = kScanTile / kScanThreads;  // consecutive counts per thread
  constexpr int kWarps = kScanThreads / 32;
  __shared__ uint64_t s_w[kWarps];
  __shared__ uint64_t s_excl;
  __shared__ uint32_t s_tile;
  __shared__ bool s_last;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned int* counters = reinterpret_cast<unsigned int*>(state + nblk);  // claim, done
  if (tid == 0) s_tile = atomicAdd(&counters[0], 1u);
  __syncthreads();
  const int tile = (int)s_tile;
  const int64_t base = (int64_t)tile * kScanTile + (int64_t)tid * kItems;
  uint32_t v[kItems];
  if (base + kItems <= S) {
    const uint4* src = reinterpret_cast<const uint4*>(a + base);
#pragma unroll
    for (int q = 0; q < kItems / 4; ++q) {
      const uint4 x = src[q];
      v[4 * q] = x.x, v[4 * q + 1] = x.y, v[4 * q + 2] = x.z, v[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kItems; ++k) v[k] = base + k < S ? a[base + k] : 0u;
  }
  uint64_t sum = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) sum += v[k];
  uint64_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_w[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    // publish this tile's sum, then the first warp reads the status words of
    // the 32 tiles before it at once, window after window, until one holds an
    // inclusive prefix (or tile 0 is reached)
    uint64_t agg = 0;
    for (int w = 0; w < kWarps; ++w) agg += s_w[w];
    volatile uint64_t* st = state;
    if (lane == 0) st[tile] = (tile == 0 ? kScanPrefix : kScanAggregate) | agg;
    uint64_t excl = 0;
    int top = tile - 1;  // newest tile not yet summed
    int spins = 0;
    while (top >= 0) {
      const int j = top - lane;
      uint64_t w = kScanPrefix;  // before tile 0: prefix 0
      if (j >= 0) w = st[j];
      // the window is usable up to the first tile still unpublished
      const unsigned pending = __ballot_sync(0xffffffffu, w == 0u);
      const unsigned pref = __ballot_sync(0xffffffffu, (w & kScanPrefix) != 0u);
      const int first_pending = pending ? __ffs(pending) - 1 : 32;
      const int first_pref = pref ? __ffs(pref) - 1 : 32;
      const int take = min(first_pending, first_pref + 1);  // lanes [0, take) summed
      uint64_t v = lane < take ? (w & kScanValue) : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      excl += v;
      if (first_pref < first_pending) break;  // reached an inclusive prefix
      top -= take;
      if (take == 0) {
        if (++spins > kLbSpinLimit) {  // never expected: tiles before are running
          if (lane == 0) set_status(hdr, GFTORF_ERR_TIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    if (lane == 0) {
      if (tile != 0) st[tile] = kScanPrefix | (excl + agg);
      s_excl = excl;
    }
  }
  __syncthreads();
  uint64_t run = s_excl + incl - sum;
  for (int w = 0; w < wid; ++w) run += s_w[w];
  if (base + kItems <= S) {
    uint4* dst = reinterpret_cast<uint4*>(a + base);
#pragma unroll
    for (int q = 0; q < kItems / 4; ++q) {
      uint4 x;
      x.x = (uint32_t)run; run += v[4 * q];
      x.y = (uint32_t)run; run += v[4 * q + 1];
      x.z = (uint32_t)run; run += v[4 * q + 2];
      x.w = (uint32_t)run; run += v[4 * q + 3];
      dst[q] = x;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      if (base + k < S) a[base + k] = (uint32_t)run;
      run += v[k];
    }
  }
  // the last CTA to finish sees every tile's offsets
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&counters[1], 1u) == (unsigned)(nblk - 1);
  __syncthreads();
  if (!s_last || wid != 0) return;
  __threadfence();
  // chunk table by one warp: lane l takes frames l and l + 32 (at most 64)
  const uint64_t total = *reinterpret_cast<volatile uint64_t*>(&state[nblk - 1]) & kScanValue;
  const bool over = total > (uint64_t)cap;
  uint64_t fs[2], n[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int b = lane + 32 * h;
    fs[h] = b < B ? (uint64_t)__ldcg(&a[(size_t)b * N]) : total;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // the next frame's first instance
    uint64_t fe = __shfl_down_sync(0xffffffffu, fs[h], 1);
    const uint64_t wrap = __shfl_sync(0xffffffffu, h == 0 ? fs[1] : total, 0);
    if (lane == 31) fe = wrap;
    const int b = lane + 32 * h;
    n[h] = (b < B && !over) ? (fe - fs[h] + kChunk - 1) / kChunk : 0u;
  }
  uint64_t nrun = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint64_t incl = n[h];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int b = lane + 32 * h;
    if (b < B) {
      hdr->fstart[b] = (uint32_t)fs[h];
      hdr->coff[b] = (uint32_t)(nrun + incl - n[h]);
    }
    nrun += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) {
    hdr->count = (int64_t)total;
    if (over) set_status(hdr, GFTORF_ERR_CAPACITY);
    hdr->fstart[B] = (uint32_t)total;
    hdr->coff[B] = nrun <= (uint64_t)n_chunk ? (uint32_t)nrun : (uint32_t)n_chunk;
  }
}

struct ChunkPos {
  int b;
  uint32_t s, e;  // instance range of the chunk
};

__device__ __forceinline__ ChunkPos chunk_pos(const Header* hdr, int c) {
  ChunkPos p;
  int b = 0;
  while ((uint32_t)c >= hdr->coff[b + 1]) ++b;
  p.b = b;
  p.s = hdr->fstart[b] + (uint32_t)(c - (int)hdr->coff[b]) * kChunk;
  p.e = min(p.s + (uint32_t)kChunk, hdr->fstart[b + 1]);
  return p;
}

// count the tiles hit by the instances [s, e) of one chunk: corners of each
// Gaussian's part of the chunk in a difference array, then its 2D prefix
// sum; the counts are also added to the frame's per-tile totals
__global__ void __launch_bounds__(256)
    tile_count_kernel(const uint2* __restrict__ srect, const Header* __restrict__ hdr,
                      const uint32_t* __restrict__ eoff, uint32_t* __restrict__ tcnt,
                      uint32_t* __restrict__ ttot, int N, int NT, int tiles_x, int tiles_y,
                      int B) {
  extern __shared__ uint32_t D[];  // (tiles_y + 1) x (tiles_x + 1)
  __shared__ int s_r0;
  const int n_chunks = (int)hdr->coff[B];
  for (int c = blockIdx.x; c < n_chunks; c += gridDim.x) {
  const ChunkPos cp = chunk_pos(hdr, c);
  const int vis = (int)hdr->vis[cp.b];
  const uint32_t* eb = eoff + (size_t)cp.b * N;
  const int cols = tiles_x + 1, rows = tiles_y + 1;
  for (int t = threadIdx.x; t < rows * cols; t += blockDim.x) D[t] = 0;
  if (threadIdx.x < 32) {
    const int r0 = warp_upper_rank(eb, vis, cp.s, threadIdx.x);
    if (threadIdx.x == 0) s_r0 = r0;
  }
  __syncthreads();
  const uint2* rc = srect + (size_t)cp.b * N;
  diff_add_gaussians(D, cols, eb, rc, s_r0 + threadIdx.x, blockDim.x, vis, cp.s, cp.e);
  __syncthreads();
  prefix2d<false>(D, rows, cols, threadIdx.x, blockDim.x);
  __syncthreads();
  uint32_t* out = tcnt + (size_t)c * NT;
  uint32_t* tot = ttot + (size_t)cp.b * NT;
  for (int t = threadIdx.x; t < NT; t += blockDim.x) {
    const int ty = t / tiles_x, tx = t - ty * tiles_x;
    const uint32_t v = D[ty * cols + tx];
    out[t] = v;
    if (v) atomicAdd(&tot[t], v);
  }
  __syncthreads();  // D is cleared for the next chunk
  }
}

// per (frame, tile): exclusive prefix over the frame's chunks, and the tile's
// range of the batch's list: the frame's first instance, plus the totals of
// the frame's tiles before it (those of earlier CTAs summed from the
// per-tile totals, those of this CTA's 32 tiles scanned), plus nothing else
// (a frame's instances are contiguous).  A CTA covers 32 tiles (lanes,
// coalesced rows) and splits the frame's chunks into 8 consecutive segments
// (warps): segment sums, then per-segment rescan.  Lists that overflowed
// the capacity are left empty.
__global__ void __launch_bounds__(256)
    tile_colscan_kernel(uint32_t* __restrict__ tcnt, const uint32_t* __restrict__ ttot,
                        uint2* __restrict__ ranges, const Header* __restrict__ hdr, int NT,
                        int64_t cap) {
  __shared__ uint32_t s_seg[8][32];
  __shared__ uint32_t s_pre[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t0 = blockIdx.x * 32, t = t0 + lane;
  const int b = blockIdx.y;
  const uint32_t c0 = hdr->coff[b], n = hdr->coff[b + 1] - c0;
  const uint32_t seg = (n + 7) / 8;
  const uint32_t s0 = c0 + min(n, (uint32_t)w * seg), s1 = c0 + min(n, (uint32_t)(w + 1) * seg);
  uint32_t pre = 0;  // instances of the frame's tiles [0, t0)
  for (int i = threadIdx.x; i < t0; i += blockDim.x) pre += ttot[(size_t)b * NT + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
  if (lane == 0) s_pre[w] = pre;
  uint32_t sum = 0;
  if (t < NT) {
#pragma unroll 4
    for (uint32_t c = s0; c < s1; ++c) sum += tcnt[(size_t)c * NT + t];
  }
  s_seg[w][lane] = sum;
  __syncthreads();
  uint32_t run = 0;
  for (int ww = 0; ww < w; ++ww) run += s_seg[ww][lane];
  if (t < NT) {
#pragma unroll 4
    for (uint32_t c = s0; c < s1; ++c) {
      const uint32_t v = tcnt[(size_t)c * NT + t];
      tcnt[(size_t)c * NT + t] = run;
      run += v;
    }
  }
  if (w == 7) {  // run: the tile's total
    uint32_t incl = t < NT ? run : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (t < NT) {
      uint32_t base = hdr->fstart[b];
      for (int ww = 0; ww < 8; ++ww) base += s_pre[ww];
      const uint64_t st = (uint64_t)base + incl - run, en = st + run;
      const bool over = hdr->count > cap;
      const uint64_t c = (uint64_t)cap;  // never exceeded when not over
      ranges[(size_t)b * NT + t] =
          over ? make_uint2(0u, 0u) : make_uint2((uint32_t)min(st, c), (uint32_t)min(en, c));
    }
  }
}

// Stable scatter of one chunk.  Warp w owns the instance sub-range
// [s + w kChunk/nw, ...).  Its per-tile counts come from the corners of its
// Gaussians' parts (as in tile_count); each tile's cursor for warp w starts
// at tile base + chunk prefix + earlier warps' counts.  Then the warp takes
// its Gaussians 32 at a time (depth order) and their instances in the
// sub-range 32 at a time, one per lane in list order (a lane finds its
// Gaussian by counting the Gaussians that start at or before its slot);
// lanes that share a tile take consecutive places in lane order, ranked by
// __match_any_sync; the row-major index in the rectangle is split into (row,
// column) with an approximate float reciprocal (relative error near 2^-23:
// for indices below 50000 the quotient is off by far less than one) and an
// exact one-step correction.
__device__ __forceinline__ void scatter_chunk(int c, const uint32_t* __restrict__ sorted_ids,
                                              const uint2* __restrict__ srect,
                                              const Header* __restrict__ hdr,
                                              const uint32_t* __restrict__ eoff,
                                              const uint32_t* __restrict__ tcnt,
                                              const uint2* __restrict__ ranges,
                                              uint32_t* __restrict__ values, int N, int NT,
                                              int tiles_x, int tiles_y, int64_t cap) {
  extern __shared__ uint32_t cur[];  // [warps][(tiles_y + 1) x (tiles_x + 1)]
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ChunkPos cp = chunk_pos(hdr, c);
  const int vis = (int)hdr->vis[cp.b];
  const uint32_t* eb = eoff + (size_t)cp.b * N;
  const uint32_t* ids = sorted_ids + (size_t)cp.b * N;
  const uint2* rc = srect + (size_t)cp.b * N;
  const int cols = tiles_x + 1, rows = tiles_y + 1, A = rows * cols;
  for (int i = threadIdx.x; i < nw * A; i += blockDim.x) cur[i] = 0;
  const uint32_t per = kChunk / nw;
  const uint32_t sw = cp.s + (uint32_t)w * per;
  const uint32_t ew = min(sw + per, cp.e);
  const bool active = sw < ew;
  const int rw = active ? warp_upper_rank(eb, vis, sw, lane) : 0;
  uint32_t* D = cur + (size_t)w * A;
  __syncthreads();
  // phase 1: this warp's tile counts
  if (active) {
    diff_add_gaussians(D, cols, eb, rc, rw + lane, 32, vis, sw, ew);
    __syncwarp();
    prefix2d<true>(D, rows, cols, lane, 32);
  }
  __syncthreads();
  // phase 2: cursors
  const uint32_t* cc = tcnt + (size_t)c * NT;
  const uint2* to = ranges + (size_t)cp.b * NT;
  for (int t = threadIdx.x; t < NT; t += blockDim.x) {
    const int ty = t / tiles_x, idx = t + ty;  // ty * cols + (t - ty * tiles_x)
    uint32_t run = to[t].x + cc[t];
    for (int ww = 0; ww < nw; ++ww) {
      const uint32_t v = cur[(size_t)ww * A + idx];
      cur[(size_t)ww * A + idx] = run;
      run += v;
    }
  }
  __syncthreads();
  if (!active) return;
  // phase 3: the batch's instances 32 at a time, one per lane, in list order
  __shared__ int4 s_g[8][32];     // per warp and non-empty Gaussian: lo - start, width, index, corner
  __shared__ float s_inv[8][32];  // 1 / width
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t capu = cap < (int64_t)0xFFFFFFFF ? (uint32_t)cap : 0xFFFFFFFFu;
  // the next batch's offsets, indices and rectangles are loaded while the
  // current one is written
  uint32_t eo_n = 0, g_n = 0;
  uint2 pr_n = make_uint2(0, 0);
  if (rw + lane < vis) {
    eo_n = eb[rw + lane];
    g_n = ids[rw + lane];
    pr_n = rc[rw + lane];
  }
  for (int rb = rw;; rb += 32) {
    const int r = rb + lane;
    const uint32_t eo = eo_n, g = g_n;
    const uint2 pr = pr_n;
    const bool ok = r < vis && eo < ew;
    if (r + 32 < vis) {
      eo_n = eb[r + 32];
      g_n = ids[r + 32];
      pr_n = rc[r + 32];
    }
    const unsigned take = __ballot_sync(0xffffffffu, ok);
    if (!take) break;
    int x0, y0, x1, y1;
    unpack_rect(pr, x0, y0, x1, y1);
    const int wd = ok ? x1 - x0 : 1;
    const uint32_t n_all = ok ? (uint32_t)(wd * (y1 - y0)) : 0u;
    const uint32_t lo = ok ? max(sw, eo) - eo : 0u;
    const uint32_t n = ok ? min(ew, eo + n_all) - eo - lo : 0u;
    // slots [start, start + n) of the batch's instances are this Gaussian's
    uint32_t incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t start = incl - n;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const bool ne = n > 0u;
    const unsigned nem = __ballot_sync(0xffffffffu, ne);
    if (ne) {  // non-empty Gaussians packed in order: their starts increase strictly
      const int ci = __popc(nem & lt);
      s_g[w][ci] = make_int4((int)lo - (int)start, wd, (int)g, x0 | (y0 << 16));
      s_inv[w][ci] = rcp_approx((float)wd);
    }
    __syncwarp();
    int carry = -1;  // packed index of the Gaussian owning the slot before the window
    for (uint32_t base = 0; base < total; base += 32) {
      // bit s: a Gaussian starts at slot base + s
      const uint32_t rel = start - base;
      const unsigned sb = __reduce_or_sync(0xffffffffu, ne && rel < 32u ? 1u << rel : 0u);
      const int jj = carry + __popc(sb & (lt | (1u << lane)));
      carry += __popc(sb);  // lane 31's jj
      const uint32_t i = base + (uint32_t)lane;
      int idx = -1, gj = 0;
      if (i < total) {
        const int4 q = s_g[w][jj];
        const float inv = s_inv[w][jj];
        const int local = q.x + (int)i;
        int ky = (int)((float)local * inv);
        int kx = local - ky * q.y;
        if (kx < 0) {
          --ky;
          kx += q.y;
        } else if (kx >= q.y) {
          ++ky;
          kx -= q.y;
        }
        idx = ((q.w >> 16) + ky) * cols + (q.w & 0xFFFF) + kx;
        gj = q.z;
      }
      const bool act = (unsigned)idx < (unsigned)A;
      const unsigned am = __ballot_sync(0xffffffffu, act);
      if (act) {
        // lanes of one tile take consecutive places, in slot (= depth) order
        const unsigned peers = __match_any_sync(am, idx);
        const uint32_t p = D[idx] + __popc(peers & lt);
        __syncwarp(am);
        if ((peers >> lane) == 1u) D[idx] = p + 1u;
        if (p < capu) values[p] = (uint32_t)gj;
      }
      __syncwarp();
    }
    if (take != 0xffffffffu) break;
  }
}

// CTAs loop over the batch's chunks (the grid is what fits on the GPU at
// once; the chunk count is known only on the device)
__global__ void __launch_bounds__(256, 8)
    tile_scatter_kernel(const uint32_t* __restrict__ sorted_ids,
                        const uint2* __restrict__ srect,
                        const Header* __restrict__ hdr,
                        const uint32_t* __restrict__ eoff,
                        const uint32_t* __restrict__ tcnt,
                        const uint2* __restrict__ ranges,
                        uint32_t* __restrict__ values, int N, int NT,
                        int tiles_x, int tiles_y, int B, int64_t cap) {
  const int n_chunks = (int)hdr->coff[B];
  for (int c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    scatter_chunk(c, sorted_ids, srect, hdr, eoff, tcnt, ranges, values, N, NT, tiles_x,
                  tiles_y, cap);
    __syncthreads();  // the cursors are cleared for the next chunk
  }
}


__global__ void export_keys_kernel(const uint2* __restrict__ ranges,
                                   const uint32_t* __restrict__ values,
                                   const uint32_t* __restrict__ zkey,
                                   uint64_t* __restrict__ keys, int N, int NT) {
  const int t = blockIdx.x, b = blockIdx.y;
  const uint2 r = ranges[(size_t)b * NT + t];
  const uint64_t hi = ((uint64_t)b * NT + t) << 32;
  for (uint32_t i = r.x + threadIdx.x; i < r.y; i += blockDim.x)
    keys[i] = hi | zkey[(size_t)b * N + values[i]];
}

}  // namespace

// look-back region: 64 words of per-pass tile counters, then one status word
// per (pass, frame, tile, digit)
constexpr size_t kLbCounters = 64;
size_t lb_bytes(const Layout& L) {
  return (kLbCounters + (size_t)4 * L.B * (L.n_dblk > 0 ? L.n_dblk : 1) * 256) * 4;
}

void launch_footprints(const Layout& L, const float* u, const float* v,
                       const int32_t* radius, const float* z,
                       unsigned char* ws, cudaStream_t st) {
  if (L.N == 0) return;
  dim3 grid((L.N + 255) / 256, L.B);
  footprint_kernel<<<grid, 256, 0, st>>>(
      u, v, radius, z, at<Header>(ws, L.off_header), at<uint2>(ws, L.off_rect),
      at<uint32_t>(ws, L.off_zkey), L.N, L.TW, L.TH, L.tiles_x, L.tiles_y);
  count_launches(1);
}

// CTAs of a kernel that loops over the batch's chunks: as many as are
// resident at once (at most one per chunk the capacity allows)
template <typename KernelT>
int chunk_grid(KernelT kernel, int threads, size_t smem, int n_chunk) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  return max(1, min(n_chunk, per_sm * sm_count()));
}

void launch_binning(const Layout& L, unsigned char* ws, cudaStream_t st) {
  static PerDeviceOnce attr;
  attr.run([] {  // per-CTA tile counters may exceed the default 48 KB
    // (at most 50000 counters of 4 bytes per CTA: see the dims checks)
    return cudaFuncSetAttribute(tile_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024) == cudaSuccess &&
           cudaFuncSetAttribute(tile_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024) == cudaSuccess;
  });
  auto* hdr = at<Header>(ws, L.off_header);
  auto* zkey = at<uint32_t>(ws, L.off_zkey);
  auto* k0 = at<uint32_t>(ws, L.off_zkey2);
  auto* k1 = k0 + (size_t)L.B * L.N;
  auto* i0 = at<uint32_t>(ws, L.off_ids);
  auto* i1 = at<uint32_t>(ws, L.off_ids2);
  auto* lb = at<uint32_t>(ws, L.off_dhist);     // pass tile counters, then status words
  auto* ghist = at<uint32_t>(ws, L.off_dtot);   // [frame][pass][digit] totals -> bases
  auto* rect = at<const uint2>(ws, L.off_rect);
  auto* srect = at<uint2>(ws, L.off_srect);
  auto* ecnt = at<uint32_t>(ws, L.off_ecnt);
  auto* bsum = at<uint64_t>(ws, L.off_bsum);
  auto* tcnt = at<uint32_t>(ws, L.off_tcnt);
  auto* ttot = at<uint32_t>(ws, L.off_toff);
  auto* ranges = at<uint2>(ws, L.off_ranges);
  auto* values = at<uint32_t>(ws, L.off_values);
  const uint32_t* sorted = i1;
  if (L.N == 0) {
    cudaMemsetAsync(ranges, 0, (size_t)L.B * L.NT * sizeof(uint2), st);
    return;
  }
  // 1. depth sort: zkey -> (k0,i0) -> (k1,i1) -> (k0,i0) -> (k1,i1); the
  // digit totals of all passes, then one look-back kernel per pass
  const uint32_t* kin = zkey;
  const uint32_t* iin = nullptr;
  uint32_t* kout[2] = {k0, k1};
  uint32_t* iout[2] = {i0, i1};
  // the look-back words and the digit totals are adjacent: one memset
  cudaMemsetAsync(lb, 0, L.off_dtot + (size_t)L.B * 1024 * 4 - L.off_dhist, st);
  dsort_hist_kernel<<<dim3(L.n_dblk, L.B), kSortThreads, 0, st>>>(zkey, L.N, ghist);
  dsort_bases_kernel<<<L.B * 4, 256, 0, st>>>(ghist, ttot, L.B * L.NT, bsum, L.n_scan + 1);
  for (int pass = 0; pass < 4; ++pass) {
    dsort_pass_kernel<<<L.B * L.n_dblk, kSortThreads, 0, st>>>(
        kin, iin, kout[pass & 1], iout[pass & 1], L.N, L.B, pass, L.n_dblk, ghist,
        lb + kLbCounters, lb + pass, hdr, pass == 3 ? rect : nullptr,
        pass == 3 ? srect : nullptr, pass == 3 ? ecnt : nullptr);
    kin = kout[pass & 1];
    iin = iout[pass & 1];
  }
  // 2. emission offsets of the depth-ordered Gaussians (their tile counts
  // written by the last pass), chunk table
  emission_scan_kernel<<<L.n_scan, kScanThreads, 0, st>>>(ecnt, (int64_t)L.B * L.N, bsum, L.n_scan, hdr,
                                                 L.B, L.N, L.cap, L.n_chunk);
  // 3. per-chunk tile counts and per-tile totals; per-frame column scan and
  // tile ranges
  const size_t corners = (size_t)(L.tiles_x + 1) * (L.tiles_y + 1) * 4;
  tile_count_kernel<<<chunk_grid(tile_count_kernel, 256, corners, L.n_chunk), 256, corners, st>>>(srect, hdr, ecnt, tcnt, ttot, L.N, L.NT,
                                                     L.tiles_x, L.tiles_y, L.B);
  tile_colscan_kernel<<<dim3((L.NT + 31) / 32, L.B), 256, 0, st>>>(tcnt, ttot, ranges, hdr,
                                                                   L.NT, L.cap);
  // 4. stable scatter
  const int nw = L.scatter_warps;
  tile_scatter_kernel<<<chunk_grid(tile_scatter_kernel, nw * 32, (size_t)nw * corners, L.n_chunk),
                        nw * 32, (size_t)nw * corners, st>>>(
      sorted, srect, hdr, ecnt, tcnt, ranges, values, L.N, L.NT, L.tiles_x, L.tiles_y, L.B,
      L.cap);
  count_launches(10);
}

void launch_export_keys(const Layout& L, uint64_t* keys, unsigned char* ws,
                        cudaStream_t st) {
  dim3 g(L.NT, L.B);
  export_keys_kernel<<<g, 128, 0, st>>>(
      at<const uint2>(ws, L.off_ranges), at<const uint32_t>(ws, L.off_values),
      at<const uint32_t>(ws, L.off_zkey), keys, L.N, L.NT);
  count_launches(1);
}

}  // namespace gftorf
