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

// Copies src[0..n) (global, uint32) into dst (shared) with 16-byte vector
// loads for the aligned body, several loads in flight per thread.
__device__ __forceinline__ void stage_u32(uint32_t* dst, const uint32_t* __restrict__ src, int n) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const uintptr_t a = reinterpret_cast<uintptr_t>(src);
  int head = (int)(((16 - (a & 15)) & 15) >> 2);
  if ((a & 3) != 0) head = n;  // not even 4-byte aligned: all scalar
  if (head > n) head = n;
  for (int i = tid; i < head; i += nt) dst[i] = __ldg(src + i);
  const int nv = (n - head) >> 2;
  const uint4* s4 = reinterpret_cast<const uint4*>(src + head);
  int i = tid;
  for (; i + 3 * nt < nv; i += 4 * nt) {
    uint4 v0 = __ldg(s4 + i), v1 = __ldg(s4 + i + nt), v2 = __ldg(s4 + i + 2 * nt),
          v3 = __ldg(s4 + i + 3 * nt);
    uint32_t* d = dst + head;
    d[4 * i + 0] = v0.x; d[4 * i + 1] = v0.y; d[4 * i + 2] = v0.z; d[4 * i + 3] = v0.w;
    int j = i + nt;
    d[4 * j + 0] = v1.x; d[4 * j + 1] = v1.y; d[4 * j + 2] = v1.z; d[4 * j + 3] = v1.w;
    j += nt;
    d[4 * j + 0] = v2.x; d[4 * j + 1] = v2.y; d[4 * j + 2] = v2.z; d[4 * j + 3] = v2.w;
    j += nt;
    d[4 * j + 0] = v3.x; d[4 * j + 1] = v3.y; d[4 * j + 2] = v3.z; d[4 * j + 3] = v3.w;
  }
  for (; i < nv; i += nt) {
    uint4 v = __ldg(s4 + i);
    uint32_t* d = dst + head + 4 * i;
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  }
  for (int k = head + 4 * nv + tid; k < n; k += nt) dst[k] = __ldg(src + k);
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
  for (uint64_t i = e0 + gtid; i < e1; i += gsz) {
    const uint32_t v = __ldg(idx + i);
    if (v >= WH) { ++drop; continue; }
    uint32_t y, x;
    dw.divmod(v, y, x);
    sx += x; sy += y; sn += 1;
    if (pacbed) atomicAdd(pacbed + v, 1ull);
  }
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
// Per-frame integer sums, one thread per frame, events of the CTA's frames
// staged in shared memory with vector loads (Eq. 4 on linear-index EER).
constexpr int kComFrames = 256;
constexpr int kComStage = 16384;

__global__ void __launch_bounds__(kThreads) k_com(const uint32_t* __restrict__ idx, uint64_t n_idx,
                                                  const uint64_t* __restrict__ off, uint32_t F,
                                                  uint32_t WH, DivMod dw,
                                                  const long long* __restrict__ totals,
                                                  double cx_h, double cy_h, float zscale,
                                                  long long* sums, float* com, float2* z,
                                                  uint32_t* st) {
  extern __shared__ uint32_t ev[];
  __shared__ unsigned long long s_lo, s_hi;
  __shared__ float s_cfx, s_cfy;
  __shared__ long long s_cix, s_ciy;
  const uint32_t f0 = blockIdx.x * kComFrames;
  const uint32_t f = f0 + threadIdx.x;
  const bool have = f < F;
  uint64_t lo = 0, hi = 0;
  bool bad = false;
  if (have) frame_range(off, f, n_idx, lo, hi, bad);
  if (threadIdx.x == 0) {
    s_lo = ~0ull; s_hi = 0;
    // centre: integer part (exact) + fractional part (float), from double
    double cx = cx_h, cy = cy_h;
    if (totals) {
      const long long n = totals[2];
      cx = n ? (double)totals[0] / (double)n : 0.0;
      cy = n ? (double)totals[1] / (double)n : 0.0;
    }
    const double rx = rint(cx), ry = rint(cy);
    s_cix = (long long)rx; s_ciy = (long long)ry;
    s_cfx = (float)(cx - rx); s_cfy = (float)(cy - ry);
  }
  __syncthreads();
  if (have && hi > lo) {
    atomicMin(&s_lo, (unsigned long long)lo);
    atomicMax(&s_hi, (unsigned long long)hi);
  }
  if (bad) st_or(st, EER4D_ST_OFFSETS);
  __syncthreads();
  const uint64_t E0 = s_lo, E1 = s_hi;
  unsigned long long sx = 0, sy = 0, sn = 0;
  uint32_t drop = 0;
  for (uint64_t base = E0; base < E1; base += kComStage) {
    const int cnt = (int)min((uint64_t)kComStage, E1 - base);
    __syncthreads();
    stage_u32(ev, idx + base, cnt);
    __syncthreads();
    if (have) {
      const uint64_t a = lo > base ? lo : base;
      const uint64_t b = hi < base + cnt ? hi : base + cnt;
      uint32_t px = 0, py = 0, pn = 0;
      for (uint64_t i = a; i < b; ++i) {
        const uint32_t v = ev[i - base];
        if (v >= WH) { ++drop; continue; }
        uint32_t y, x;
        dw.divmod(v, y, x);
        px += x; py += y; ++pn;
      }
      sx += px; sy += py; sn += pn;
    }
  }
  if (have) {
    sums[f] = (long long)sx;
    sums[F + f] = (long long)sy;
    sums[2 * (size_t)F + f] = (long long)sn;
    float ox = 0.f, oy = 0.f;
    if (sn) {
      const long long dx = (long long)sx - (long long)sn * s_cix;
      const long long dy = (long long)sy - (long long)sn * s_ciy;
      ox = (float)dx / (float)sn - s_cfx;
      oy = (float)dy / (float)sn - s_cfy;
    }
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

// ---------------------------------------------------------------- a4 -------
// Bin + crop + densify.  A CTA owns TF consecutive frames (aligned to
// multiples of TF in the scan) and all P_pad pixels: it counts into a shared
// tile of packed 16-bit counters (two frames per word), then writes
// counts[p][f] as fp16 rows.  No global atomics; every (p, f) of the chunk is
// written exactly once, zeros included.
constexpr int kScatStage = 8192;
constexpr int kMaxFrameEvents = 65535;

__global__ void __launch_bounds__(kThreads) k_scatter(
    const uint32_t* __restrict__ idx, uint64_t n_idx, const uint64_t* __restrict__ off,
    uint64_t first, uint64_t nfr, uint32_t WH, DivMod dw, const int16_t* __restrict__ lutx,
    const int16_t* __restrict__ luty, const int32_t* __restrict__ lut2, int pw, int P_pad, int TF,
    uint64_t NR, __half* counts, uint32_t* st) {
  extern __shared__ uint32_t smem[];
  uint32_t* tile = smem;                                  // [P_pad][TF/2]
  uint32_t* ev = smem + (size_t)P_pad * (TF / 2);         // [kScatStage]
  __shared__ unsigned long long s_lo, s_hi;
  const int TW = TF / 2;
  const uint64_t T0 = (first / TF) * TF;
  const uint64_t tf0 = T0 + (uint64_t)blockIdx.x * TF;    // global frame of tile column 0
  const uint64_t end = first + nfr;
  for (int i = threadIdx.x; i < P_pad * TW; i += blockDim.x) tile[i] = 0u;
  if (threadIdx.x == 0) { s_lo = ~0ull; s_hi = 0; }
  __syncthreads();
  // frame ranges of the tile's frames that belong to this chunk
  bool bad = false;
  for (int j = threadIdx.x; j < TF; j += blockDim.x) {
    const uint64_t g = tf0 + j;
    if (g < first || g >= end) continue;
    uint64_t lo, hi;
    bool b;
    frame_range(off, g - first, n_idx, lo, hi, b);
    bad |= b;
    if (hi - lo > kMaxFrameEvents) { bad = true; st_or(st, EER4D_ST_OVERFLOW); }
    if (hi > lo) { atomicMin(&s_lo, (unsigned long long)lo); atomicMax(&s_hi, (unsigned long long)hi); }
  }
  if (bad) st_or(st, EER4D_ST_OFFSETS);
  __syncthreads();
  const uint64_t E0 = s_lo, E1 = s_hi;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  uint32_t drop = 0;
  for (uint64_t base = E0; base < E1; base += kScatStage) {
    const int cnt = (int)min((uint64_t)kScatStage, E1 - base);
    __syncthreads();
    stage_u32(ev, idx + base, cnt);
    __syncthreads();
    for (int j = warp; j < TF; j += nw) {
      const uint64_t g = tf0 + j;
      if (g < first || g >= end) continue;
      uint64_t lo, hi;
      bool b;
      frame_range(off, g - first, n_idx, lo, hi, b);
      if (hi - lo > kMaxFrameEvents) hi = lo + kMaxFrameEvents;
      const uint64_t a = lo > base ? lo : base;
      const uint64_t e = hi < base + cnt ? hi : base + cnt;
      const uint32_t inc = 1u << (16 * (j & 1));
      uint32_t* col = tile + (j >> 1);
      for (uint64_t i = a + lane; i < e; i += 32) {
        const uint32_t v = ev[i - base];
        if (v >= WH) { ++drop; continue; }
        uint32_t y, x;
        dw.divmod(v, y, x);
        const int u = __ldg(lutx + x), vv = __ldg(luty + y);
        if ((u | vv) < 0) continue;
        const int p = __ldg(lut2 + vv * pw + u);
        if (p < 0) continue;
        atomicAdd(col + (size_t)p * TW, inc);
      }
    }
  }
  __syncthreads();
  // write counts[p][tf0 .. tf0+TF) for frames inside the chunk
  uint32_t over = 0;
  const bool full = tf0 >= first && tf0 + TF <= end && tf0 + TF <= NR;
  for (int i = threadIdx.x; i < P_pad * TW; i += blockDim.x) {
    const int p = i / TW, w = i - p * TW;
    const uint32_t word = tile[i];
    const uint32_t c0 = word & 0xffffu, c1 = word >> 16;
    over += (c0 > 2048u) + (c1 > 2048u);
    const __half h0 = __ushort2half_rn((unsigned short)c0);
    const __half h1 = __ushort2half_rn((unsigned short)c1);
    const uint64_t g = tf0 + 2 * w;
    __half* dst = counts + (size_t)p * NR + g;
    if (full) {
      *reinterpret_cast<__half2*>(dst) = __halves2half2(h0, h1);
    } else {
      if (g >= first && g < end && g < NR) dst[0] = h0;
      if (g + 1 >= first && g + 1 < end && g + 1 < NR) dst[1] = h1;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    drop += __shfl_xor_sync(0xffffffffu, drop, o);
    over += __shfl_xor_sync(0xffffffffu, over, o);
  }
  if (lane == 0) {
    if (drop) { st_or(st, EER4D_ST_RANGE); st_add(st, 1, drop); }
    if (over) { st_or(st, EER4D_ST_OVERFLOW); st_add(st, 2, over); }
  }
}

}  // namespace

int scatter_tf(int P_pad) {
  int tf = 256;
  while (tf > 2 && (size_t)P_pad * tf * 2 > 80 * 1024) tf >>= 1;
  return tf;
}

cudaError_t launch_validate(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx,
                            const uint64_t* off, uint64_t n_frames, int64_t* pacbed,
                            int64_t* totals, uint32_t* st, cudaStream_t s) {
  const uint64_t work = n_frames > n_idx ? n_frames : n_idx;
  uint64_t blocks = (work + kThreads - 1) / kThreads;
  if (blocks > 152 * 16) blocks = 152 * 16;
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
  const size_t sm = kComStage * sizeof(uint32_t);
  cudaError_t e = ensure_smem((const void*)k_com, sm);
  if (e != cudaSuccess) return e;
  const float zscale = (float)(p->g.dalpha_raw_rad / p->g.lambda_A);
  stage_begin(p, EER4D_STAGE_COM, s);
  k_com<<<(F + kComFrames - 1) / kComFrames, kThreads, sm, s>>>(
      idx, n_idx, off, F, p->g.det_w * p->g.det_h, p->dw,
      reinterpret_cast<const long long*>(totals), cx, cy, zscale,
      reinterpret_cast<long long*>(sums), com, z, st);
  count_launches(1);
  stage_end(p, EER4D_STAGE_COM, s);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx,
                           const uint64_t* off, uint64_t first, uint64_t n, __half* counts,
                           uint32_t* st, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int TF = scatter_tf(p->P_pad);
  const size_t sm = (size_t)p->P_pad * (TF / 2) * 4 + kScatStage * 4;
  cudaError_t e = ensure_smem((const void*)k_scatter, sm);
  if (e != cudaSuccess) return e;
  const uint64_t T0 = (first / TF) * TF;
  const uint64_t tiles = (first + n - T0 + TF - 1) / TF;
  stage_begin(p, EER4D_STAGE_SCATTER, s);
  k_scatter<<<(unsigned)tiles, kThreads, sm, s>>>(
      idx, n_idx, off, first, n, p->g.det_w * p->g.det_h, p->dw, p->d_lutx, p->d_luty, p->d_lut2,
      (int)p->g.pw, p->P_pad, TF, (uint64_t)p->F, counts, st);
  count_launches(1);
  stage_end(p, EER4D_STAGE_SCATTER, s);
  return cudaGetLastError();
}
