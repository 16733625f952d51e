// Run-length-encoded EER (Sec. II, Fig. 1c): within a frame the hits are in
// ascending linear index and each run is the distance from the previous hit
// (run 0: from pixel 0).  Re-coding to linear-index encoding is an O(C)
// segmented inclusive prefix sum: idx_j = run_0 + ... + run_j.
//
// One warp per frame: the frame's runs are read 32 at a time (coalesced), a
// warp inclusive scan adds them up, the carry moves to the next 32.  The
// scan runs in 64 bits so a sum beyond the uint32 index range is detected.
#include "common.cuh"

namespace {

constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_rle_decode(const uint32_t* runs, uint64_t n, const uint64_t* __restrict__ off,
                 uint64_t n_frames, uint32_t* idx, uint32_t* st) {
  const uint64_t f = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (f >= n_frames) return;  // whole warp
  const uint64_t a = off[f], b = off[f + 1];
  const uint64_t lo = a < n ? a : n;
  const uint64_t t = b > lo ? b : lo;
  const uint64_t hi = t < n ? t : n;
  if (lane == 0 && ((b < a) || (b > n) || (a > n))) st_or(st, EER4D_ST_OFFSETS);
  unsigned long long carry = 0ull;
  bool over = false;
  for (uint64_t base = lo; base < hi; base += 32) {  // uniform trip count per warp
    const uint64_t i = base + lane;
    const unsigned long long r = i < hi ? (unsigned long long)runs[i] : 0ull;
    const unsigned long long s = carry + warp_incl_scan_u64(r, lane);
    if (i < hi) {
      const bool big = s > 0xFFFFFFFFull;
      over |= big;
      idx[i] = big ? 0xFFFFFFFFu : (uint32_t)s;
    }
    carry = __shfl_sync(0xffffffffu, s, 31);
  }
  if (over) st_or(st, EER4D_ST_RANGE);
}

}  // namespace

cudaError_t launch_rle_decode(const uint32_t* runs, uint64_t n, const uint64_t* off,
                              uint64_t n_frames, uint32_t* idx, uint32_t* st, cudaStream_t s) {
  if (n_frames == 0) return cudaSuccess;
  const uint64_t blocks = (n_frames + kWarpsPerBlock - 1) / kWarpsPerBlock;
  k_rle_decode<<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(runs, n, off, n_frames, idx, st);
  count_launches(1);
  return cudaGetLastError();
}
