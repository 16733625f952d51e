// Virtual detectors from linear-index EER (Table 1: operations that scale with
// the number of counts): per frame, the number of events in each of n_rings
// annuli about the pattern centre, the annular bright-field, annular
// dark-field or radial-sum images of a pixelated detector, in O(C).
//
// Ring j holds the raw pixels (x, y) with r_j^2 <= (x - cx)^2 + (y - cy)^2 <
// r_{j+1}^2, every square and sum in double with round-to-nearest and no
// fused multiply-add, so an independent float64 evaluation in the same order
// decides every pixel the same way.  A first kernel writes the ring of every
// detector pixel into an int8 table (W*H bytes of scratch); the second walks
// the frames, one warp per frame, and looks each event up in that table.
#include "common.cuh"

namespace {

constexpr int kFramesPerBlock = 32;
constexpr int kWarps = 8;

struct Rings {
  int n;                              // rings
  double r2[EER4D_MAX_RINGS + 1];     // squared radii, ascending
};

__global__ void k_ring_table(uint32_t W, uint32_t H, const long long* __restrict__ totals,
                             double cx_h, double cy_h, Rings R, signed char* lut) {
  double cx = cx_h, cy = cy_h;
  if (totals) {
    const long long n = totals[2];
    cx = n ? (double)totals[0] / (double)n : 0.0;
    cy = n ? (double)totals[1] / (double)n : 0.0;
  }
  const size_t WH = (size_t)W * H;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < WH;
       i += (size_t)gridDim.x * blockDim.x) {
    const double dx = __dsub_rn((double)(i % W), cx);
    const double dy = __dsub_rn((double)(i / W), cy);
    const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    int ring = -1;
    if (r2 >= R.r2[0]) {
      for (int j = 0; j < R.n; ++j)
        if (r2 < R.r2[j + 1]) {
          ring = j;
          break;
        }
    }
    lut[i] = (signed char)ring;
  }
}

// Block: kFramesPerBlock consecutive frames, kWarps warps taking frames in
// turn; counts go to shared memory [ring][frame] and leave as rows of 32
// consecutive frames (128-byte stores).
__global__ void __launch_bounds__(kWarps * 32)
    k_ring_counts(const uint32_t* __restrict__ idx, uint64_t n_idx,
                  const uint64_t* __restrict__ off, uint64_t n_frames, uint32_t WH,
                  const signed char* __restrict__ lut, int n_rings, int32_t* out, uint32_t* st) {
  extern __shared__ int cnt[];  // [n_rings][kFramesPerBlock]
  const uint64_t f0 = (uint64_t)blockIdx.x * kFramesPerBlock;
  for (int i = threadIdx.x; i < n_rings * kFramesPerBlock; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bool bad = false, range = false;
  for (int fl = warp; fl < kFramesPerBlock; fl += kWarps) {
    const uint64_t f = f0 + fl;
    if (f >= n_frames) break;
    const uint64_t a = off[f], b = off[f + 1];
    const uint64_t lo = a < n_idx ? a : n_idx;
    const uint64_t t = b > lo ? b : lo;
    const uint64_t hi = t < n_idx ? t : n_idx;
    bad |= (b < a) || (b > n_idx) || (a > n_idx);
    for (uint64_t i = lo + lane; i < hi; i += 32) {
      const uint32_t v = idx[i];
      if (v >= WH) {
        range = true;
        continue;
      }
      const int ring = lut[v];
      if (ring >= 0) atomicAdd(&cnt[ring * kFramesPerBlock + fl], 1);
    }
  }
  if (lane == 0 && bad) st_or(st, EER4D_ST_OFFSETS);
  if (range) st_or(st, EER4D_ST_RANGE);
  __syncthreads();
  for (int i = threadIdx.x; i < n_rings * kFramesPerBlock; i += blockDim.x) {
    const int j = i / kFramesPerBlock, fl = i - j * kFramesPerBlock;
    const uint64_t f = f0 + fl;
    if (f < n_frames) out[(size_t)j * n_frames + f] = cnt[i];
  }
}

}  // namespace

size_t vdet_scratch_bytes(const eer4d_plan* p) { return (size_t)p->g.det_w * p->g.det_h; }

cudaError_t launch_virtual_detectors(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx,
                                     const uint64_t* off, uint64_t n_frames, const double* radii,
                                     int n_rings, const int64_t* totals, double cx, double cy,
                                     void* scratch, int32_t* out, uint32_t* st, cudaStream_t s) {
  Rings R;
  R.n = n_rings;
  for (int j = 0; j <= n_rings; ++j) R.r2[j] = radii[j] * radii[j];
  for (int j = n_rings + 1; j <= EER4D_MAX_RINGS; ++j) R.r2[j] = 0.0;
  signed char* lut = static_cast<signed char*>(scratch);
  const uint32_t W = p->g.det_w, H = p->g.det_h;
  k_ring_table<<<608, 256, 0, s>>>(W, H, reinterpret_cast<const long long*>(totals), cx, cy, R, lut);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_frames == 0) return e;
  const uint64_t blocks = (n_frames + kFramesPerBlock - 1) / kFramesPerBlock;
  const size_t sm = sizeof(int) * (size_t)n_rings * kFramesPerBlock;
  k_ring_counts<<<(unsigned)blocks, kWarps * 32, sm, s>>>(idx, n_idx, off, n_frames, W * H, lut,
                                                         n_rings, out, st);
  count_launches(1);
  return cudaGetLastError();
}
