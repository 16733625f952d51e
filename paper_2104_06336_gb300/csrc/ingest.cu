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
// tile of packed 16-bit counters (two frames per word, rows padded by one word
// so the pixels of a frame fall in different banks), then writes
// counts[p][f] as fp16, four frames per 8-byte store.  No global atomics;
// every (p, f) of the chunk is written exactly once, zeros included.  The
// tile is kept small (<= 48 KB) so several CTAs overlap their phases.
constexpr int kScatStage = 4096;
constexpr int kMaxFrameEvents = 65535;

__global__ void __launch_bounds__(kThreads) k_scatter(
    const uint32_t* __restrict__ idx, uint64_t n_idx, const uint64_t* __restrict__ off,
    uint64_t first, uint64_t nfr, uint32_t WH, DivMod dw, const int16_t* __restrict__ lutx,
    const int16_t* __restrict__ luty, const int32_t* __restrict__ lut2, int pw, int P_pad, int TF,
    uint64_t NR, __half* counts, uint32_t* st) {
  extern __shared__ uint32_t smem[];
  __shared__ uint32_t s_lo[128], s_hi[128];  // event range of each tile frame, relative to E0
  __shared__ unsigned long long s_e0, s_e1;
  const int TW = TF / 2;
  const int TP = TW + 1;
  uint32_t* tile = smem;                     // [P_pad][TP]
  uint32_t* ev = smem + (size_t)P_pad * TP;  // [kScatStage]
  const uint64_t T0 = (first / TF) * TF;
  const uint64_t tf0 = T0 + (uint64_t)blockIdx.x * TF;  // global frame of tile column 0
  const uint64_t end = first + nfr;
  // frames j of the tile inside the chunk: [j0, j1)
  const int j0 = tf0 < first ? (int)(first - tf0) : 0;
  const int j1 = tf0 + TF > end ? (int)(end - tf0) : TF;
  {
    uint4* t4 = reinterpret_cast<uint4*>(tile);  // P_pad * TP is a multiple of 4 (P_pad % 16 == 0)
    const int n4 = P_pad * TP / 4;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) t4[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (threadIdx.x == 0) { s_e0 = ~0ull; s_e1 = 0; }
  __syncthreads();
  bool bad = false;
  uint64_t lo = 0, hi = 0;
  if (threadIdx.x >= j0 && threadIdx.x < j1) {
    bool b;
    frame_range(off, tf0 + threadIdx.x - first, n_idx, lo, hi, b);
    bad |= b;
    if (hi - lo > kMaxFrameEvents) { bad = true; hi = lo + kMaxFrameEvents; st_or(st, EER4D_ST_OVERFLOW); }
    if (hi > lo) { atomicMin(&s_e0, (unsigned long long)lo); atomicMax(&s_e1, (unsigned long long)hi); }
  }
  if (bad) st_or(st, EER4D_ST_OFFSETS);
  __syncthreads();
  const uint64_t E0 = s_e0, E1 = s_e1;
  if (threadIdx.x < TF) {  // 32-bit event offsets relative to E0 (a tile spans < 2^32 events)
    const bool in = threadIdx.x >= j0 && threadIdx.x < j1 && hi > lo;
    s_lo[threadIdx.x] = in ? (uint32_t)(lo - E0) : 0u;
    s_hi[threadIdx.x] = in ? (uint32_t)(hi - E0) : 0u;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  uint32_t drop = 0;
  const uint32_t nev = E1 > E0 ? (uint32_t)(E1 - E0) : 0u;
  for (uint32_t base = 0; base < nev; base += kScatStage) {
    const int cnt = (int)min((uint32_t)kScatStage, nev - base);
    __syncthreads();
    stage_u32(ev, idx + E0 + base, cnt);
    __syncthreads();
    for (int j = j0 + warp; j < j1; j += nw) {
      const uint32_t a = max(s_lo[j], base), e = min(s_hi[j], base + (uint32_t)cnt);
      const uint32_t inc = 1u << (16 * (j & 1));
      uint32_t* col = tile + (j >> 1);
      for (uint32_t i = a + lane; i < e; i += 32) {
        const uint32_t v = ev[i - base];
        if (v >= WH) { ++drop; continue; }
        uint32_t y, x;
        dw.divmod(v, y, x);
        const int u = __ldg(lutx + x), vv = __ldg(luty + y);
        if ((u | vv) < 0) continue;
        const int p = __ldg(lut2 + vv * pw + u);
        if (p < 0) continue;
        atomicAdd(col + p * TP, inc);
      }
    }
  }
  __syncthreads();
  // write counts[p][tf0 + 4w .. tf0 + 4w + 3] (two tile words, four fp16) per lane
  uint32_t over = 0;
  const bool full = j0 == 0 && j1 == TF;
  const int QW = TW / 2;  // 8-byte groups per pixel row
  for (int i = threadIdx.x; i < P_pad * QW; i += blockDim.x) {
    const int p = i / QW, w = i - p * QW;
    const uint32_t w0 = tile[p * TP + 2 * w], w1 = tile[p * TP + 2 * w + 1];
    const uint32_t c0 = w0 & 0xffffu, c1 = w0 >> 16, c2 = w1 & 0xffffu, c3 = w1 >> 16;
    over += (c0 > 2048u) + (c1 > 2048u) + (c2 > 2048u) + (c3 > 2048u);
    const __half2 h01 = __halves2half2(__ushort2half_rn((unsigned short)c0), __ushort2half_rn((unsigned short)c1));
    const __half2 h23 = __halves2half2(__ushort2half_rn((unsigned short)c2), __ushort2half_rn((unsigned short)c3));
    __half* dst = counts + (size_t)p * NR + tf0 + 4 * w;
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

// frames per scatter tile: a multiple of 4 (8-byte count stores), at most
// 128, with the padded tile P_pad x (TF/2 + 1) words within 48 KB
int scatter_tf(int P_pad) {
  int tf = 128;
  while (tf > 4 && (size_t)P_pad * (tf / 2 + 1) * 4 > 48 * 1024) tf >>= 1;
  return tf;
}

cudaError_t launch_validate(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx,
                            const uint64_t* off, uint64_t n_frames, int64_t* pacbed,
                            int64_t* totals, uint32_t* st, cudaStream_t s) {
  const uint64_t work = n_frames > n_idx / 16 ? n_frames : n_idx / 16;
  uint64_t blocks = (work + kThreads - 1) / kThreads;
  if (blocks > 152 * 8) blocks = 152 * 8;
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
  const size_t sm = (size_t)p->P_pad * (TF / 2 + 1) * 4 + kScatStage * 4;
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
