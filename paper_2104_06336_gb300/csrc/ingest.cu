// Event ingest kernels (Sec. II linear-index EER; Table 1 bin, crop, centre of
// mass and sum of all frames; Eq. 4).
//
// Every kernel re-derives each frame's event range defensively:
//   lo = min(off[f], n_idx), hi = min(max(off[f+1], lo), n_idx)
// so corrupt offsets never cause an out-of-bounds read; they set
// EER4D_ST_OFFSETS instead.  Indices >= det_w*det_h are dropped and counted.
#include "common.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void frame_range(const uint64_t* off, uint64_t f, uint64_t n_idx,
                                            uint64_t& lo, uint64_t& hi, bool& bad) {
  const uint64_t a = off[f], b = off[f + 1];
  lo = a < n_idx ? a : n_idx;
  uint64_t t = b > lo ? b : lo;
  hi = t < n_idx ? t : n_idx;
  bad = (b < a) || (b > n_idx) || (a > n_idx);
}

// ---------------------------------------------------------------- a1 -------
// Offsets check, index range check, integer totals and optional PACBED.
__global__ void __launch_bounds__(kThreads) k_validate(const uint32_t* __restrict__ idx,
                                                       uint64_t n_idx,
                                                       const uint64_t* __restrict__ off,
                                                       uint64_t n_frames, uint32_t WH, DivMod dw,
                                                       unsigned long long* pacbed,
                                                       unsigned long long* totals, uint32_t* st) {
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t gsz = (uint64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (uint64_t f = gtid; f < n_frames; f += gsz) {
    uint64_t lo, hi;
    bool b;
    frame_range(off, f, n_idx, lo, hi, b);
    bad |= b;
  }
  if (bad) st_or(st, EER4D_ST_OFFSETS);
  // events referenced by the frames: [min lo, max hi) == [off[0], off[n]) for valid data
  uint64_t e0 = off[0] < n_idx ? off[0] : n_idx;
  uint64_t e1 = off[n_frames] < n_idx ? off[n_frames] : n_idx;
  if (e1 < e0) e1 = e0;
  unsigned long long sx = 0, sy = 0, sn = 0;
  uint32_t drop = 0;
  auto one = [&](uint32_t v) {
    if (v >= WH) { ++drop; return; }
    uint32_t y, x;
    dw.divmod(v, y, x);
    sx += x; sy += y; sn += 1;
    if (pacbed) atomicAdd(pacbed + v, 1ull);
  };
  // scalar head up to a 16-byte boundary, then 4 x uint4 per thread in flight
  uint64_t head = e0;
  const uintptr_t a = reinterpret_cast<uintptr_t>(idx + e0);
  if ((a & 3) == 0) head = e0 + (((16 - (a & 15)) & 15) >> 2);
  else head = e1;
  if (head > e1) head = e1;
  for (uint64_t i = e0 + gtid; i < head; i += gsz) one(__ldg(idx + i));
  const uint64_t nv = (e1 - head) >> 2;
  const uint4* v4 = reinterpret_cast<const uint4*>(idx + head);
  uint64_t i = gtid;
  for (; i + 3 * gsz < nv; i += 4 * gsz) {
    const uint4 q0 = __ldg(v4 + i), q1 = __ldg(v4 + i + gsz), q2 = __ldg(v4 + i + 2 * gsz),
                q3 = __ldg(v4 + i + 3 * gsz);
    one(q0.x); one(q0.y); one(q0.z); one(q0.w);
    one(q1.x); one(q1.y); one(q1.z); one(q1.w);
    one(q2.x); one(q2.y); one(q2.z); one(q2.w);
    one(q3.x); one(q3.y); one(q3.z); one(q3.w);
  }
  for (; i < nv; i += gsz) {
    const uint4 q = __ldg(v4 + i);
    one(q.x); one(q.y); one(q.z); one(q.w);
  }
  for (uint64_t k = head + 4 * nv + gtid; k < e1; k += gsz) one(__ldg(idx + k));
  if (totals) {
    sx = warp_sum_ll(sx); sy = warp_sum_ll(sy); sn = warp_sum_ll(sn);
    if ((threadIdx.x & 31) == 0 && sn) {
      atomicAdd(totals + 0, sx);
      atomicAdd(totals + 1, sy);
      atomicAdd(totals + 2, sn);
    }
  }
  for (int o = 16; o > 0; o >>= 1) drop += __shfl_xor_sync(0xffffffffu, drop, o);
  if ((threadIdx.x & 31) == 0 && drop) {
    st_or(st, EER4D_ST_RANGE);
    st_add(st, 1, drop);
  }
}

// ---------------------------------------------------------------- a2 -------
// Per-frame integer sums (Eq. 4 on linear-index EER), one thread per frame.
// A thread reads its frame's events straight from global memory, 16-byte
// vector loads with four in flight (a frame's events are contiguous, so the
// 32 frames of a warp cover one contiguous stretch of the event array and
// every fetched sector is used); no shared staging and no block barrier
// before the sums.  Thread 0 computes the centre meanwhile.
constexpr int kComThreads = 256;
// frames of at most this many events sum x and y in 32 bits (x, y < 32768)
constexpr uint64_t kComFast = 131071;

// The COM centre as an exact integer part and a float fraction (from double):
// the PACBED centre of mass from the totals, or (cx, cy) when there are none.
struct ComCentre {
  long long ix, iy;
  float fx, fy;
};
__device__ __forceinline__ ComCentre com_centre(const long long* totals, double cx, double cy) {
  if (totals) {
    const long long n = totals[2];
    cx = n ? (double)totals[0] / (double)n : 0.0;
    cy = n ? (double)totals[1] / (double)n : 0.0;
  }
  const double rx = rint(cx), ry = rint(cy);
  ComCentre c;
  c.ix = (long long)rx;
  c.iy = (long long)ry;
  c.fx = (float)(cx - rx);
  c.fy = (float)(cy - ry);
  return c;
}
// COM of one frame relative to the centre, (Sx - N round(cx)) / N - frac(cx)
// in float32 (0 for an empty frame).
__device__ __forceinline__ void com_of_frame(long long sx, long long sy, long long sn,
                                             const ComCentre& c, float& ox, float& oy) {
  ox = oy = 0.f;
  if (sn) {
    const long long dx = sx - sn * c.ix;
    const long long dy = sy - sn * c.iy;
    ox = (float)dx / (float)sn - c.fx;
    oy = (float)dy / (float)sn - c.fy;
  }
}

__global__ void __launch_bounds__(kComThreads, 8) k_com(const uint32_t* __restrict__ idx, uint64_t n_idx,
                                                     const uint64_t* __restrict__ off, uint32_t F,
                                                     uint32_t WH, DivMod dw,
                                                     const long long* __restrict__ totals,
                                                     double cx_h, double cy_h, float zscale,
                                                     long long* sums, float* com, float2* z,
                                                     uint32_t* st) {
  __shared__ ComCentre s_c;
  if (threadIdx.x == 0) s_c = com_centre(totals, cx_h, cy_h);
  const uint32_t f = blockIdx.x * kComThreads + threadIdx.x;
  unsigned long long sx = 0, sy = 0, sn = 0;
  uint32_t drop = 0;
  if (f < F) {
    uint64_t lo, hi;
    bool bad;
    frame_range(off, f, n_idx, lo, hi, bad);
    if (bad) st_or(st, EER4D_ST_OFFSETS);
    uint32_t px = 0, py = 0, pn = 0;
    auto one = [&](uint32_t v) {
      if (v >= WH) { ++drop; return; }
      uint32_t y, x;
      dw.divmod(v, y, x);
      px += x; py += y; ++pn;
    };
    uint64_t i = lo;
    if (hi - lo > kComFast) {
      // a frame too long for 32-bit sums (never at detector doses): 64-bit
      for (; i < hi; ++i) {
        const uint32_t v = __ldg(idx + i);
        if (v >= WH) { ++drop; continue; }
        uint32_t y, x;
        dw.divmod(v, y, x);
        sx += x; sy += y; ++sn;
      }
    } else if ((reinterpret_cast<uintptr_t>(idx) & 15) == 0) {
      for (; i < hi && (i & 3); ++i) one(__ldg(idx + i));
      for (; i + 16 <= hi; i += 16) {
        const uint4* q = reinterpret_cast<const uint4*>(idx + i);
        const uint4 a0 = __ldg(q), a1 = __ldg(q + 1), a2 = __ldg(q + 2), a3 = __ldg(q + 3);
        one(a0.x); one(a0.y); one(a0.z); one(a0.w);
        one(a1.x); one(a1.y); one(a1.z); one(a1.w);
        one(a2.x); one(a2.y); one(a2.z); one(a2.w);
        one(a3.x); one(a3.y); one(a3.z); one(a3.w);
      }
      for (; i + 4 <= hi; i += 4) {
        const uint4 a0 = __ldg(reinterpret_cast<const uint4*>(idx + i));
        one(a0.x); one(a0.y); one(a0.z); one(a0.w);
      }
    }
    for (; i < hi; ++i) one(__ldg(idx + i));
    sx += px; sy += py; sn += pn;
  }
  __syncthreads();  // the centre
  if (f < F) {
    sums[f] = (long long)sx;
    sums[F + f] = (long long)sy;
    sums[2 * (size_t)F + f] = (long long)sn;
    float ox, oy;
    com_of_frame((long long)sx, (long long)sy, (long long)sn, s_c, ox, oy);
    com[f] = ox;
    com[F + f] = oy;
    if (z) z[f] = make_float2(ox * zscale, oy * zscale);
  }
  for (int o = 16; o > 0; o >>= 1) drop += __shfl_xor_sync(0xffffffffu, drop, o);
  if ((threadIdx.x & 31) == 0 && drop) {
    st_or(st, EER4D_ST_RANGE);
    st_add(st, 1, drop);
  }
}

// COM maps from per-frame sums [3][F] already formed (by the scatter pass of
// ssb_accumulate_com): the same centre and arithmetic as k_com.
__global__ void __launch_bounds__(kComThreads) k_com_from_sums(const long long* __restrict__ sums,
                                                               uint32_t F,
                                                               const long long* __restrict__ totals,
                                                               double cx_h, double cy_h,
                                                               float zscale, float* com, float2* z) {
  __shared__ ComCentre s_c;
  if (threadIdx.x == 0) s_c = com_centre(totals, cx_h, cy_h);
  __syncthreads();
  const uint32_t f = blockIdx.x * kComThreads + threadIdx.x;
  if (f >= F) return;
  float ox, oy;
  com_of_frame(sums[f], sums[F + f], sums[2 * (size_t)F + f], s_c, ox, oy);
  com[f] = ox;
  com[F + f] = oy;
  if (z) z[f] = make_float2(ox * zscale, oy * zscale);
}

// ---------------------------------------------------------------- a4 -------
// Bin + crop + densify.  A persistent CTA takes tiles of TF consecutive frames
// (aligned to multiples of TF in the scan) and all P_pad pixels: it counts
// into a shared tile of packed 16-bit counters (two frames per word, rows
// padded by one word so the pixels of a frame fall in different banks), then
// writes counts[p][f] as fp16, four frames per 8-byte store.  No global
// atomics; every (p, f) of the chunk is written exactly once, zeros included.
// Events are read straight from global memory, a warp per four frames with its
// lanes on consecutive events (128-byte loads, eight in flight per lane).
// The frame offsets of a CTA's next tile are loaded one tile ahead (threads
// below TF keep them in registers), so their latency overlaps a whole tile.
// The pixel of an event comes from the binning tables x -> u, y -> v and
// (v, u) -> kept pixel, copied once per CTA into shared memory (one divide
// by det_w and three shared loads, no L2 round trip per event); detectors
// whose tables do not fit use the raw-pixel table (or the three tables) in
// global memory.
constexpr int kMaxFrameEvents = 65535;

#ifndef EER4D_SCATTER_MINB
#define EER4D_SCATTER_MINB 2
#endif
// SUMS: the same pass also forms each frame's COM sums (Sx, Sy, N over its
// in-range events; Eq. 4) into sums[3][F] and adds them to totals[3] (the
// PACBED centre), in the tiles of pixel chunk 0; events past the first
// 65535 of a frame (EER4D_ST_OVERFLOW) are counted in neither.
template <bool SUMS>
__global__ void __launch_bounds__(kThreads, SUMS ? 3 : EER4D_SCATTER_MINB) k_scatter(
    const uint32_t* __restrict__ idx, uint64_t n_idx, const uint64_t* __restrict__ off,
    uint64_t first, uint64_t nfr, uint32_t W, uint32_t H, DivMod dw,
    const int16_t* __restrict__ lutp, const int16_t* __restrict__ lutx,
    const int16_t* __restrict__ luty, const int32_t* __restrict__ lut2, int pw, int ph, int P_pad,
    int TF, int PC, DivMod nch, uint32_t ntiles, int tab_smem, uint64_t NR, __half* counts,
    long long* sums, unsigned long long* totals, uint64_t F, uint32_t* st) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long s_lo[128];  // event range of each tile frame
  __shared__ uint32_t s_n[128];
  __shared__ uint32_t s_maxev;              // most events in one frame of the tile
  const uint32_t WH = W * H;
  const int TW = TF / 2;
  const int TP = TW + 1;
  uint32_t* tile = smem;  // [PC][TP]: the pixels [p0, p0 + PC) of the tile
  int16_t* tx = reinterpret_cast<int16_t*>(smem + (size_t)PC * TP);  // [W], [H], [ph*pw]
  int16_t* ty = tx + W;
  int16_t* t2 = ty + H;
  if (tab_smem) {
    for (uint32_t i = threadIdx.x; i < W; i += blockDim.x) tx[i] = lutx[i];
    for (uint32_t i = threadIdx.x; i < H; i += blockDim.x) ty[i] = luty[i];
    for (int i = threadIdx.x; i < pw * ph; i += blockDim.x) t2[i] = (int16_t)lut2[i];
  }
  // kept pixel of raw index v (< W*H); (x, y) are v's detector coordinates
  // when the tables or SUMS needed them
  auto pixel = [&](uint32_t v, uint32_t& x, uint32_t& y) -> int {
    if (tab_smem) {
      dw.divmod(v, y, x);
      const int u = tx[x], vv = ty[y];
      if ((u | vv) < 0 || !EER4D_IN_RANGE(vv * pw + u, pw * ph, st)) return -1;
      return t2[vv * pw + u];
    }
    if (SUMS || !lutp) dw.divmod(v, y, x);
    if (lutp) return __ldg(lutp + v);
    const int u = __ldg(lutx + x), vv = __ldg(luty + y);
    return (u | vv) < 0 ? -1 : __ldg(lut2 + vv * pw + u);
  };
  unsigned long long tsx = 0, tsy = 0, tsn = 0;  // lane 0: this warp's share of the totals
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  uint32_t drop = 0, over = 0;
  const uint64_t T0 = (first / TF) * TF;
  const uint64_t end = first + nfr;
  const int QW = TW / 2;  // 8-byte groups per pixel row (a power of two)
  const int qs = __ffs(QW) - 1;
  // threads < TF: raw offsets off[f], off[f+1] of their frame of the next
  // tile, loaded one tile ahead so the load latency overlaps a whole tile
  uint64_t na = 0, nb = 0;
  auto tile_frames = [&](uint32_t tt, uint64_t& tf0_, int& j0_, int& j1_) {
    uint32_t ft_, ch_;
    nch.divmod(tt, ft_, ch_);
    tf0_ = T0 + (uint64_t)ft_ * TF;
    j0_ = tf0_ < first ? (int)(first - tf0_) : 0;
    j1_ = tf0_ + TF > end ? (int)(end - tf0_) : TF;
  };
  if (threadIdx.x < TF && blockIdx.x < ntiles) {
    uint64_t tf0_;
    int j0_, j1_;
    tile_frames(blockIdx.x, tf0_, j0_, j1_);
    if ((int)threadIdx.x >= j0_ && (int)threadIdx.x < j1_) {
      const uint64_t f = tf0_ + threadIdx.x - first;
      na = off[f];
      nb = off[f + 1];
    }
  }
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // tile t: frames of frame tile t / NCH, pixels of chunk t % NCH (the
    // chunks of one frame tile are neighbours in t, so its events are read
    // from L2 after the first chunk)
    uint32_t ft, ch;
    nch.divmod(t, ft, ch);
    const int p0 = (int)ch * PC;
    const int pc = P_pad - p0 < PC ? P_pad - p0 : PC;
    const uint64_t tf0 = T0 + (uint64_t)ft * TF;  // global frame of tile column 0
    // frames j of the tile inside the chunk: [j0, j1)
    const int j0 = tf0 < first ? (int)(first - tf0) : 0;
    const int j1 = tf0 + TF > end ? (int)(end - tf0) : TF;
    __syncthreads();  // the previous tile is written out
    if (threadIdx.x == 0) s_maxev = 0;
    {
      uint4* t4 = reinterpret_cast<uint4*>(tile);  // PC * TP is a multiple of 4 (PC % 16 == 0)
      const int n4 = PC * TP / 4;
      for (int i = threadIdx.x; i < n4; i += blockDim.x) t4[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    if (threadIdx.x < TF) {
      uint64_t lo = 0, hi = 0;
      bool b = false;
      if (threadIdx.x >= j0 && threadIdx.x < j1) {
        // frame_range on the offsets loaded a tile ahead
        const uint64_t a = na, bb = nb;
        lo = a < n_idx ? a : n_idx;
        const uint64_t tt2 = bb > lo ? bb : lo;
        hi = tt2 < n_idx ? tt2 : n_idx;
        b = (bb < a) || (bb > n_idx) || (a > n_idx);
        if (hi - lo > kMaxFrameEvents) { b = true; hi = lo + kMaxFrameEvents; st_or(st, EER4D_ST_OVERFLOW); }
        if (b) st_or(st, EER4D_ST_OFFSETS);
      }
      s_lo[threadIdx.x] = lo;
      s_n[threadIdx.x] = (uint32_t)(hi - lo);
      if (hi > lo) atomicMax(&s_maxev, (uint32_t)(hi - lo));
      // the next tile's offsets, consumed one tile later
      const uint32_t tn = t + gridDim.x;
      na = nb = 0;
      if (tn < ntiles) {
        uint64_t tf0_;
        int j0_, j1_;
        tile_frames(tn, tf0_, j0_, j1_);
        if ((int)threadIdx.x >= j0_ && (int)threadIdx.x < j1_) {
          const uint64_t f = tf0_ + threadIdx.x - first;
          na = off[f];
          nb = off[f + 1];
        }
      }
    }
    __syncthreads();
    // a warp takes four frames at a time (j, j + nw, j + 2 nw, j + 3 nw) and
    // issues the loads of all four before using any (eight in flight per lane)
    for (int jg = j0 + warp; jg < j1; jg += 4 * nw) {
      uint64_t lo4[4];
      uint32_t n4[4], nmax = 0;
      uint32_t fsx[SUMS ? 4 : 1], fsy[SUMS ? 4 : 1], fsn[SUMS ? 4 : 1];
#pragma unroll
      for (int f = 0; f < (SUMS ? 4 : 1); ++f) fsx[f] = fsy[f] = fsn[f] = 0u;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int j = jg + f * nw;
        lo4[f] = j < j1 ? s_lo[j] : 0;
        n4[f] = j < j1 ? s_n[j] : 0u;
        nmax = n4[f] > nmax ? n4[f] : nmax;
      }
      for (uint32_t k = lane; k < nmax; k += 64) {
        uint32_t v[8];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          v[2 * f] = k < n4[f] ? __ldg(idx + lo4[f] + k) : WH;
          v[2 * f + 1] = k + 32 < n4[f] ? __ldg(idx + lo4[f] + k + 32) : WH;
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const int j = jg + f * nw;
          const uint32_t inc = 1u << (16 * (j & 1));
          uint32_t* col = tile + (j >> 1);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t kk = k + 32 * h;
            if (kk >= n4[f]) continue;
            const uint32_t e = v[2 * f + h];
            if (e >= WH) { ++drop; continue; }
            uint32_t ex = 0u, ey = 0u;
            const int pp = pixel(e, ex, ey) - p0;
            if constexpr (SUMS) { fsx[f] += ex; fsy[f] += ey; fsn[f] += 1u; }
            if ((unsigned)pp < (unsigned)pc && EER4D_IN_RANGE(pp * TP + (j >> 1), PC * TP, st))
              atomicAdd(col + pp * TP, inc);
          }
        }
      }
      if constexpr (SUMS) {
        // the four frames' sums (32-bit: < 65536 events of x, y < 65536), once per frame
        if (p0 == 0) {
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            const uint32_t a = __reduce_add_sync(0xffffffffu, fsx[f]);
            const uint32_t b = __reduce_add_sync(0xffffffffu, fsy[f]);
            const uint32_t c = __reduce_add_sync(0xffffffffu, fsn[f]);
            const int j = jg + f * nw;
            if (lane == 0 && j < j1 && EER4D_IN_RANGE(tf0 + j, F, st)) {
              const uint64_t g = tf0 + j;  // frame of the dataset
              sums[g] = a;
              sums[F + g] = b;
              sums[2 * F + g] = c;
              tsx += a;
              tsy += b;
              tsn += c;
            }
          }
        }
      }
    }
    __syncthreads();
    // write counts[p][tf0 + 4w .. tf0 + 4w + 3] (two tile words, four fp16) per lane
    const bool full = j0 == 0 && j1 == TF;
    const bool small = s_maxev < 1024u;
    // with every count below 1024, OR-ing 0x6400 (fp16 1024.0) into a 16-bit
    // count n gives the fp16 of 1024 + n exactly; subtracting 1024 gives n
    const __half2 k1024 = __floats2half2_rn(1024.f, 1024.f);
    for (int i = threadIdx.x; i < pc * QW; i += blockDim.x) {
      const int p = i >> qs, w = i & (QW - 1);
      const uint32_t w0 = tile[p * TP + 2 * w], w1 = tile[p * TP + 2 * w + 1];
      __half2 h01, h23;
      if (small) {
        const uint32_t m0 = w0 | 0x64006400u, m1 = w1 | 0x64006400u;
        h01 = __hsub2(*reinterpret_cast<const __half2*>(&m0), k1024);
        h23 = __hsub2(*reinterpret_cast<const __half2*>(&m1), k1024);
      } else {
        const uint32_t c0 = w0 & 0xffffu, c1 = w0 >> 16, c2 = w1 & 0xffffu, c3 = w1 >> 16;
        over += (c0 > 2048u) + (c1 > 2048u) + (c2 > 2048u) + (c3 > 2048u);
        h01 = __halves2half2(__ushort2half_rn((unsigned short)c0), __ushort2half_rn((unsigned short)c1));
        h23 = __halves2half2(__ushort2half_rn((unsigned short)c2), __ushort2half_rn((unsigned short)c3));
      }
      if (!EER4D_IN_RANGE((long long)(p0 + p) * (long long)NR + (long long)(tf0 + 4 * w) + 3,
                          (long long)P_pad * (long long)NR, st))
        continue;
      __half* dst = counts + (size_t)(p0 + p) * NR + tf0 + 4 * w;
      if (full) {
        uint2 pk;
        pk.x = *reinterpret_cast<const uint32_t*>(&h01);
        pk.y = *reinterpret_cast<const uint32_t*>(&h23);
        *reinterpret_cast<uint2*>(dst) = pk;
      } else {
        const __half hv[4] = {__low2half(h01), __high2half(h01), __low2half(h23), __high2half(h23)};
        for (int k = 0; k < 4; ++k) {
          const int j = 4 * w + k;
          if (j >= j0 && j < j1) dst[k] = hv[k];
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    drop += __shfl_xor_sync(0xffffffffu, drop, o);
    over += __shfl_xor_sync(0xffffffffu, over, o);
  }
  if (lane == 0) {
    if (drop) { st_or(st, EER4D_ST_RANGE); st_add(st, 1, drop); }
    if (over) { st_or(st, EER4D_ST_OVERFLOW); st_add(st, 2, over); }
    if (SUMS && tsn) {
      atomicAdd(totals + 0, tsx);
      atomicAdd(totals + 1, tsy);
      atomicAdd(totals + 2, tsn);
    }
  }
}

}  // namespace

// frames per scatter tile: a multiple of 4 (8-byte count stores), at most
// 128, with the padded tile P_pad x (TF/2 + 1) words within the tile budget
#ifndef EER4D_SCATTER_TILE_KB
#define EER4D_SCATTER_TILE_KB 40
#endif
constexpr size_t kScatterTabBytes = 64 * 1024;  // largest binning tables kept in shared memory

// Frames per scatter tile: 32 (64-byte count rows) unless tuned; the pixels
// are split into chunks whose padded tile PC x (TF/2 + 1) words fits the tile
// budget (a crop larger than the budget is counted chunk by chunk, each chunk
// re-reading the tile's events, from L2).
int scatter_tf(int P_pad) {
  (void)P_pad;
  return 32;
}

int scatter_pc(int P_pad, int TF) {
  int pc = (int)((size_t)EER4D_SCATTER_TILE_KB * 1024 / ((size_t)(TF / 2 + 1) * 4)) / 16 * 16;
  if (pc < 16) pc = 16;
  return pc < P_pad ? pc : P_pad;
}

cudaError_t launch_validate(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx,
                            const uint64_t* off, uint64_t n_frames, int64_t* pacbed,
                            int64_t* totals, uint32_t* st, cudaStream_t s) {
  const uint64_t work = n_frames > n_idx / 16 ? n_frames : n_idx / 16;
  uint64_t blocks = (work + kThreads - 1) / kThreads;
  // SMs x resident CTAs: one full wave, no partial second wave
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_validate, kThreads, 0);
  const uint64_t wave = (uint64_t)nsm * (occ > 0 ? occ : 1);
  if (blocks > wave) blocks = wave;
  if (blocks == 0) blocks = 1;
  stage_begin(p, EER4D_STAGE_VALIDATE, s);
  k_validate<<<(unsigned)blocks, kThreads, 0, s>>>(
      idx, n_idx, off, n_frames, p->g.det_w * p->g.det_h, p->dw,
      reinterpret_cast<unsigned long long*>(pacbed), reinterpret_cast<unsigned long long*>(totals),
      st);
  count_launches(1);
  stage_end(p, EER4D_STAGE_VALIDATE, s);
  return cudaGetLastError();
}

cudaError_t launch_com(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx, const uint64_t* off,
                       int64_t* sums, float* com, float2* z, const int64_t* totals, double cx,
                       double cy, uint32_t* st, cudaStream_t s) {
  const uint32_t F = (uint32_t)p->F;
  const float zscale = (float)(p->g.dalpha_raw_rad / p->g.lambda_A);
  stage_begin(p, EER4D_STAGE_COM, s);
  k_com<<<(F + kComThreads - 1) / kComThreads, kComThreads, 0, s>>>(
      idx, n_idx, off, F, p->g.det_w * p->g.det_h, p->dw,
      reinterpret_cast<const long long*>(totals), cx, cy, zscale,
      reinterpret_cast<long long*>(sums), com, z, st);
  count_launches(1);
  stage_end(p, EER4D_STAGE_COM, s);
  return cudaGetLastError();
}

cudaError_t launch_com_from_sums(const eer4d_plan* p, const int64_t* sums, float* com, float2* z,
                                 const int64_t* totals, double cx, double cy, cudaStream_t s) {
  const uint32_t F = (uint32_t)p->F;
  const float zscale = (float)(p->g.dalpha_raw_rad / p->g.lambda_A);
  stage_begin(p, EER4D_STAGE_COM, s);
  k_com_from_sums<<<(F + kComThreads - 1) / kComThreads, kComThreads, 0, s>>>(
      reinterpret_cast<const long long*>(sums), F, reinterpret_cast<const long long*>(totals), cx,
      cy, zscale, com, z);
  count_launches(1);
  stage_end(p, EER4D_STAGE_COM, s);
  return cudaGetLastError();
}

int scatter_tf_for(const eer4d_plan* p) {
  return p->tune.scatter_tf > 0 ? p->tune.scatter_tf : scatter_tf(p->P_pad);
}

cudaError_t launch_scatter(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx,
                           const uint64_t* off, uint64_t first, uint64_t n, __half* counts,
                           uint32_t* st, cudaStream_t s, int64_t* sums, int64_t* totals) {
  if (n == 0) return cudaSuccess;
  const int TF = scatter_tf_for(p);
  const int PC = scatter_pc(p->P_pad, TF);
  const int NCH = (p->P_pad + PC - 1) / PC;
  const uint32_t W = p->g.det_w, H = p->g.det_h;
  const size_t tile = (size_t)PC * (TF / 2 + 1) * 4;
  const size_t tabs = ((size_t)W + H + (size_t)p->g.pw * p->g.ph) * 2;
  // binning tables in shared memory when they fit beside the tile (a raw-pixel
  // table in global memory otherwise, or the three global tables without it)
  const int tab_smem = tabs <= kScatterTabBytes;
  const size_t sm = tile + (tab_smem ? (tabs + 15) / 16 * 16 : 0);
  const bool with_sums = sums != nullptr;
  const void* kern = with_sums ? (const void*)k_scatter<true> : (const void*)k_scatter<false>;
  cudaError_t e = ensure_smem(kern, sm);
  if (e != cudaSuccess) return e;
  const uint64_t T0 = (first / TF) * TF;
  const uint64_t tiles = (first + n - T0 + TF - 1) / TF * NCH;
  if (tiles >= (1ull << 31)) return cudaErrorInvalidValue;  // 32-bit tile indices in the kernel
  DivMod nch;
  nch.init((uint32_t)NCH);
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, sm);
  if (occ < 1) return cudaErrorInvalidConfiguration;  // the tile does not fit shared memory
  const int cps = p->tune.scatter_ctas_per_sm > 0 && p->tune.scatter_ctas_per_sm < occ
                      ? p->tune.scatter_ctas_per_sm : occ;
  uint64_t grid = (uint64_t)nsm * cps;
  if (grid > tiles) grid = tiles;
  stage_begin(p, EER4D_STAGE_SCATTER, s);
  auto kl = with_sums ? k_scatter<true> : k_scatter<false>;
  kl<<<(unsigned)grid, kThreads, sm, s>>>(
      idx, n_idx, off, first, n, W, H, p->dw, p->d_lutp, p->d_lutx, p->d_luty, p->d_lut2,
      (int)p->g.pw, (int)p->g.ph, p->P_pad, TF, PC, nch, (uint32_t)tiles, tab_smem, (uint64_t)p->cstride,
      counts, reinterpret_cast<long long*>(sums), reinterpret_cast<unsigned long long*>(totals),
      (uint64_t)p->F, st);
  count_launches(1);
  stage_end(p, EER4D_STAGE_SCATTER, s);
  return cudaGetLastError();
}
