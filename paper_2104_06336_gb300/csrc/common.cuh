// Shared device helpers and the internal plan of libeer4d (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "eer4d.h"

#define EER4D_MAX_STAGES 16
#define EER4D_WARPS_TROTTER 8

// ---------------------------------------------------------------- complex ---
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (dir = +1) or +i (dir = -1)
__device__ __forceinline__ float2 cmul_mi(float2 a, int dir) {
  return dir > 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// ------------------------------------------------------- integer division ---
// Exact floor division of a uint32 by a runtime divisor d >= 1:
// q0 = umulhi(n, floor(2^32/d)) is q or q-1, one correction makes it exact.
struct DivMod {
  uint32_t d, m;
  __host__ void init(uint32_t div) {
    d = div;
    m = div == 1 ? 0xFFFFFFFFu : (uint32_t)((1ull << 32) / div);
  }
  __device__ __forceinline__ void divmod(uint32_t n, uint32_t& q, uint32_t& r) const {
    q = __umulhi(n, m);
    r = n - q * d;
    if (r >= d) { q += 1; r -= d; }
  }
};

// ---------------------------------------------------------------- FFT plan ---
// First factor R1 of the register four-step split N = R1 * R2 (R1 >= R2) for
// power-of-two N in [16, 1024], 0 for other lengths.
__host__ __device__ constexpr int reg_r1(int N) {
  return N == 1024 || N == 512 ? 32 : N == 256 || N == 128 ? 16 : N == 64 || N == 32 ? 8 : N == 16 ? 4 : 0;
}

// Stockham radix-decomposition of one transform length; twiddles tw[j] =
// exp(-2 pi i j / N) made on the host in double from the exact integer j.
// For the register four-step lengths, tw4[k1 * R2 + j2] = tw[j2 k1]
// (R1 = reg_r1(N) rows of R2): a thread of the first pass (fixed j2) reads
// its twiddles at constant offsets, and the lanes of a warp (consecutive j2)
// read consecutive entries.
struct FftDesc {
  int N;
  int nst;
  int radix[EER4D_MAX_STAGES];
  const float2* tw;
  const float2* tw4;  // NULL unless reg_r1(N) > 0
};

// ------------------------------------------------------------- plan state ---
struct eer4d_plan {
  eer4d_geom g;
  int precision, norm;
  int P, P_pad, P_bf, n_rows, nkx, list_max;
  // pixel shard: this plan owns the kept pixels [p_begin, p_end) of the full
  // plan's numbering (shard of n_shards; 0 of 1 for an ordinary plan)
  int shard, n_shards, p_begin, p_end;
  int F;
  long long cstride;         // row stride (elements) of the fp16 counts [P_pad][cstride]
  DivMod dw;                 // division by det_w
  // device tables (owned)
  int16_t* d_lutx;           // [det_w] binned u or -1
  int16_t* d_luty;           // [det_h] binned v or -1
  int32_t* d_lut2;           // [ph*pw] kept pixel index or -1
  int16_t* d_lutp;           // [det_h*det_w] kept pixel of each raw pixel or -1 (NULL when
                             // the detector has more than 2^24 pixels)
  short2* d_pix;             // [P_pad] (kx, ky)
  int32_t* d_bfp;            // [P_bf] kept-pixel index of each bright-field pixel (row-major)
  __half* d_dft_hi;          // split-FP16 DFT matrix along x (tile-blocked), SPLIT_FP16 plans
  __half* d_dft_lo;
  unsigned char* d_tc4_tabs;  // four-step tensor-core DFT: split factor matrices (SPLIT_FP16, 1024 columns)
  float2* d_tc4_tw;           // and its twiddles W1024^(xl kl) / 2 [32][17]
  int4* d_rows;              // [n_rows] (ky, bf kx lo, bf kx hi, p at bf lo)
  uint32_t* d_tl_bits;       // trotter membership lists at rotation 0 (NULL: none)
  uint32_t* d_tl_qp;
  int* d_tl_n;
  int* d_tl_order;           // warp tasks by decreasing list length (work-queue order)
  int tl_cap;
  float2* d_tw_y;            // [scan_ny] (+ [scan_ny] four-step layout, FftDesc)
  float2* d_tw_x;            // [scan_nx] (+ [scan_nx])
  float2* d_tw_y2;           // [2 scan_ny] (+ [2 scan_ny]; zero-padded DPC grid)
  float2* d_tw_x2;           // [2 scan_nx] (+ [2 scan_nx])
  FftDesc fy, fx, fy2, fx2;
  // streaming state of ssb_accumulate (host)
  uint64_t next_frame;
  // launch shapes chosen by eer4d_autotune / eer4d_set_tuning (0 = built-in choice)
  eer4d_tuning tune;
  // optional per-stage timing events (caller-owned cudaEvent_t), see
  // eer4d_set_stage_events
  cudaEvent_t ev_start[EER4D_N_STAGES];
  cudaEvent_t ev_stop[EER4D_N_STAGES];
};

// stage timing: records the caller's events around a launch group on the
// launching stream; counts kernel launches for eer4d_launch_count
void stage_begin(const eer4d_plan* p, int stage, cudaStream_t s);
void stage_end(const eer4d_plan* p, int stage, cudaStream_t s);
void count_launches(int n);
// EER4D_OK for cudaSuccess; otherwise records the error text for
// eer4d_last_error and returns EER4D_ECUDA.
int cuda_status(cudaError_t e);
// Raises a kernel's dynamic shared-memory limit to at least `bytes`; remembers
// what it set so repeated launches (and graph captures) make no further call.
cudaError_t ensure_smem(const void* kernel, size_t bytes);

// ---------------------------------------------------------- status helpers ---
__device__ __forceinline__ void st_or(uint32_t* st, uint32_t bits) {
  if (st) atomicOr(st, bits);
}
__device__ __forceinline__ void st_add(uint32_t* st, int word, uint32_t n) {
  if (st && n) atomicAdd(st + word, n);
}

// ---------------------------------------------------------- bounds checks ---
// Debug build (-DEER4D_CHECKS): EER4D_IN_RANGE(i, n, st) tests 0 <= i < n for
// an index derived from data or tables before the access it guards; a
// failure sets EER4D_ST_BOUNDS and the caller skips the access.  The release
// build compiles the test to `true`.
#ifdef EER4D_CHECKS
__device__ __forceinline__ bool eer4d_in_range(long long i, long long n, uint32_t* st) {
  if (i >= 0 && i < n) return true;
  st_or(st, EER4D_ST_BOUNDS);
  return false;
}
#define EER4D_IN_RANGE(i, n, st) eer4d_in_range((long long)(i), (long long)(n), (st))
#else
#define EER4D_IN_RANGE(i, n, st) true
#endif

// ------------------------------------------------------------ warp helpers ---
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_excl_scan(int v, int& total) {
  int lane = threadIdx.x & 31;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// signed frequency index of bin m of an N-point DFT (numpy fftfreq order)
__host__ __device__ __forceinline__ int freq_index(int m, int N) { return (2 * m < N) ? m : m - N; }

// ------------------------------------------------------ internal launchers ---
// (defined in the .cu files; all return cudaError_t of the launch)
cudaError_t launch_validate(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx,
                            const uint64_t* off, uint64_t n_frames, int64_t* pacbed,
                            int64_t* totals, uint32_t* st, cudaStream_t s);
cudaError_t launch_com(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx, const uint64_t* off,
                       int64_t* sums, float* com, float2* z, const int64_t* totals, double cx,
                       double cy, uint32_t* st, cudaStream_t s);
cudaError_t launch_g_slices(const eer4d_plan* p, const float2* G, const int32_t* bins, int n,
                            float2* out, cudaStream_t s);
size_t vdet_scratch_bytes(const eer4d_plan* p);
cudaError_t launch_virtual_detectors(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx,
                                     const uint64_t* off, uint64_t n_frames, const double* radii,
                                     int n_rings, const int64_t* totals, double cx, double cy,
                                     void* scratch, int32_t* out, uint32_t* st, cudaStream_t s);
cudaError_t launch_rle_decode(const uint32_t* runs, uint64_t n, const uint64_t* off,
                              uint64_t n_frames, uint32_t* idx, uint32_t* st, cudaStream_t s);
int scatter_tf_for(const eer4d_plan* p);
// sums [3][F] and totals [3] non-NULL: the same pass forms the per-frame COM
// sums of the frames [first, first + n) and adds them to totals
cudaError_t launch_scatter(const eer4d_plan* p, const uint32_t* idx, uint64_t n_idx,
                           const uint64_t* off, uint64_t first, uint64_t n, __half* counts,
                           uint32_t* st, cudaStream_t s, int64_t* sums = nullptr,
                           int64_t* totals = nullptr);
cudaError_t launch_com_from_sums(const eer4d_plan* p, const int64_t* sums, float* com, float2* z,
                                 const int64_t* totals, double cx, double cy, cudaStream_t s);
cudaError_t launch_stage1(const eer4d_plan* p, const __half* counts, float2* G, int y0, int y1,
                          cudaStream_t s);
cudaError_t launch_stage2(const eer4d_plan* p, const float2* X1, float2* G, cudaStream_t s);
cudaError_t make_dftx_tc(eer4d_plan* p);
// exp(-2 pi i k x / n), component c (0 cos, 1 -sin), from the exact integer
// phase index (k x) mod n, split as hi = fp16(w), lo = fp16(w - hi)
void dft_split_factor(int n, long long k, long long x, int c, __half* hi, __half* lo);
// four-step tensor-core DFT along x for 1024-column scans
cudaError_t make_dftx_tc4(eer4d_plan* p);
bool dftx_tc4_ok(const eer4d_plan* p);
cudaError_t launch_stage1_tc4(const eer4d_plan* p, const __half* counts, float2* X1, int y0, int y1,
                              uint32_t* st, cudaStream_t s);
cudaError_t launch_stage1_tc(const eer4d_plan* p, const __half* counts, float2* X1, int y0, int y1,
                             uint32_t* st, cudaStream_t s);
cudaError_t launch_transpose(const float2* in, float2* out, int rows, int cols, int batch,
                             cudaStream_t s);
// accumulation workspace of ssb_accumulate: fp16 counts [P_pad][F], then (at a
// 256-byte boundary) either the DFT-along-x intermediate complex64
// [nkx][Ny][P_pad], or, for plans that take the fused two-axis DFT, its ring of
// three pixel-group slabs followed (at a 256-byte boundary) by its task counters
size_t work_counts_bytes(const eer4d_plan* p);
size_t work_bytes(const eer4d_plan* p);
bool dft2_fused_ok(const eer4d_plan* p);
cudaError_t launch_wait_selftest(unsigned* ctl, uint32_t* st, cudaStream_t s);
size_t dft2_ring_bytes(const eer4d_plan* p);
size_t dft2_ctl_bytes(const eer4d_plan* p);
cudaError_t launch_dft2_fused(const eer4d_plan* p, const __half* counts, float2* ring, float2* G,
                              unsigned* ctl, uint32_t* st, cudaStream_t s);
cudaError_t launch_idpc(const eer4d_plan* p, float2* z, float* phase, double lam1, double lam2,
                        cudaStream_t s);
// complex 2D transform in place over [fy.N][fx.N], output scaled by scale
cudaError_t launch_fft2_c2c(const FftDesc& fy, const FftDesc& fx, float2* data, int dir,
                            float scale, cudaStream_t s);
size_t dpc_iterative_scratch_bytes(const eer4d_plan* p, int pad);
cudaError_t launch_dpc_iterative(const eer4d_plan* p, const float* com, double lam1, double lam2,
                                 double mu, int n_iter, int pad, void* scratch, float* phase,
                                 cudaStream_t s);
cudaError_t launch_c2r_image(const eer4d_plan* p, float2* H, float* phase, int n_cand, cudaStream_t s);
cudaError_t launch_r2c_image(const eer4d_plan* p, const float* g, float2* W, cudaStream_t s);

// trotter modes
enum { TROT_FWD = 0, TROT_GRAD = 1, TROT_VARGRAD = 2, TROT_COUNT = 3 };
cudaError_t launch_ascent(double* theta, const double* step, const double* grad, cudaStream_t s);
cudaError_t launch_adam(double* theta, const double* rate, double* state, const double* grad,
                        cudaStream_t s);
size_t trotter_batched_scratch_bytes(const eer4d_plan* const* plans, int n);
size_t trotter_lists_bytes(const eer4d_plan* p);
cudaError_t build_trotter_lists(eer4d_plan* p);
cudaError_t launch_trotter_batched(const eer4d_plan* const* plans, const float2* const* G, int n,
                                   const double* aberr, void* scratch, float* const* phase,
                                   double* var, uint32_t* st, cudaStream_t s);
size_t trotter_scratch_bytes(const eer4d_plan* p, int n_cand, int mode);
// pixel shards: this plan's share of H (scale N_R, no Gbar0) and of
// (sum G(k, 0), bright-field count); the image from summed shares
cudaError_t launch_trotter_partial(const eer4d_plan* p, const float2* G, const double* aberr,
                                   int n_cand, void* scratch, float2* H_out, double* g0_out,
                                   uint32_t* st, cudaStream_t s);
cudaError_t launch_image_from_spectrum(const eer4d_plan* p, const float2* H_in, const double* g0,
                                       int n_cand, void* scratch, float* phase_out, double* var_out,
                                       cudaStream_t s);
cudaError_t launch_trotter(const eer4d_plan* p, const float2* G, const double* aberr, int n_cand,
                           int mode, void* scratch, const float2* W, float* phase_out,
                           double* var_out, double* grad_out, int32_t* count_out, uint32_t* st,
                           cudaStream_t s);
