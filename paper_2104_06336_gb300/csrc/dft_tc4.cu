// Four-step split-FP16 tensor-core DFT along the scan x axis for scans of
// 1024 columns (Sec. IV: the scan transform of the G function written as
// complex matrix products).
//
// With x = xl + 32 xh and k = kl + 32 kh (xl, xh, kl, kh in [0, 32)):
//   X(kl + 32 kh) = sum_xl W32^(xl kh) W1024^(xl kl) [sum_xh c(xl + 32 xh) W32^(xh kl)]
// Stage A (the bracket) runs on the exact fp16 counts with the DFT-32
// factors split hi + lo: A[(b, xl)][kl] = c * Whi + c * Wlo, FP32 accumulation
// in tensor memory.  The counts are real, so A(kl) for kl = 17..31 is
// conj A(32 - kl) and only kl = 0..16 are formed.  The epilogue multiplies
// by W1024^(xl kl) (FP32, exact integer phase index) and by 1/2 (so every
// value fits fp16: |A| <= 32 * 2048), splits the result D = Dhi + Dlo into
// fp16 and stores it as the operand of stage B, which forms
//   X[(b, kl)][kh] = Dhi Whi + Dlo Whi + Dhi Wlo
// (the product Dlo Wlo, below 2^-22 relative, is dropped) for all kh.  The
// outputs X(k) for k = 0 .. 512 come from the rows kl = 0..16 directly
// (k = kl + 32 kh) or as conj X(1024 - k).
//
// Operand layouts (shared memory):
//   counts tile [b][xh][xl] fp16, one 64-byte row per (b, xh), loaded by a 3D
//     TMA copy with 64-byte swizzle: the MN-major A operand of stage A
//     (M = (b, xl), K = xh; atoms of 32 M x 8 K, 2 KB between pixels);
//   stage-B A operand [b][k][kl] fp16, k = xl (real parts) or 32 + xl
//     (imaginary parts), one 64-byte row per (b, k), kl = 0..16 used and
//     17..31 zero: MN-major, 64-byte swizzle, 4 KB between pixels;
//   factor matrices: K-major core matrices without swizzle.
// One CTA per SM takes (scan row, 8-pixel group) tasks in turn; the next
// task's counts tile is loaded by TMA while the current one computes.  Every
// mbarrier wait is bounded; on expiry the CTA sets EER4D_ST_TIMEOUT, waits
// (bounded) for its copies in flight, frees its tensor memory and returns.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kPx = 8;                  // pixels per task
constexpr int kNA = 48;                 // stage-A accumulator columns (17 complex, padded)
constexpr int kNB = 64;                 // stage-B accumulator columns (32 complex)
// tensor-memory columns: stage-A accumulators of the two 4-pixel blocks at 0
// and 64, stage-B accumulators at 128 and 192
__host__ __device__ constexpr uint32_t colA(int mb) { return (uint32_t)(64 * mb); }
__host__ __device__ constexpr uint32_t colB(int mb) { return (uint32_t)(128 + 64 * mb); }
constexpr int kThreads4 = 128;
constexpr int kTile = kPx * 32 * 64;    // 16 KB counts tile
constexpr int kFacA = kNA * 32 * 2;     // 3 KB: stage-A factors, N 48 x K 32
constexpr int kFacB = kNB * 64 * 2;     // 8 KB: stage-B factors, N 64 x K 64
constexpr int kOpB = kPx * 64 * 64;     // 32 KB: stage-B A operand (hi or lo)
constexpr int kOutPitch = 9;            // float2 per staged output row (8 pixels + 1)
constexpr int kNk = 513;                // stored K_x = 0 .. 512
// shared-memory map (bytes from a 1024-aligned base)
constexpr int kOffTile = 0;                          // 2 tiles
constexpr int kOffFac = kOffTile + 2 * kTile;        // Ahi, Alo, Bhi, Blo factors
constexpr int kOffOpB = kOffFac + 2 * kFacA + 2 * kFacB;  // hi, lo operands
constexpr int kOffOut = kOffOpB + 2 * kOpB;          // staged outputs
constexpr int kSmem4 = kOffOut + kNk * kOutPitch * 8;
constexpr int kTabBytes4 = 2 * kFacA + 2 * kFacB;    // factor tables in global memory
static_assert(kOffFac % 1024 == 0 && kOffOpB % 1024 == 0, "swizzled tiles need 1024-byte alignment");

// byte offset of element (n, k) of a K-major no-swizzle factor matrix with
// K columns (8 x 16-byte core matrices: 128 bytes between K neighbours,
// 16 K bytes between 8-row groups)
__host__ __device__ constexpr uint32_t fac_off(int n, int k, int K) {
  return (uint32_t)((n >> 3) * (K * 16) + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2);
}

// byte offset of the 16-byte chunk `chunk` of 64-byte row `row` of a
// 64-byte-swizzled tile (the row's 16-byte chunks are permuted by bits 1-2
// of the row index; tile base aligned to 512 bytes)
__device__ __forceinline__ uint32_t sw64_chunk(uint32_t row, uint32_t chunk) {
  return row * 64u + ((chunk ^ ((row >> 1) & 3u)) << 4);
}

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// 32 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Task t: pixel group g = t % n_groups (pixels 8g .. 8g+7), scan row
// y = y0 + t / n_groups.  X1: complex64 [513][Ny][P_pad].
__global__ void __launch_bounds__(kThreads4, 1)
    k_dftx_tc4(const __grid_constant__ CUtensorMap tm, const unsigned char* __restrict__ tabs,
               const float2* __restrict__ tw, float2* __restrict__ X1, int n_groups, int Ny,
               int P_pad, int y0, int ntasks, uint32_t* st) {
  extern __shared__ unsigned char sm_raw[];
  const uint32_t raw = smem_u32(sm_raw);
  unsigned char* sm = sm_raw + (((raw + 1023u) & ~1023u) - raw);
  __shared__ uint64_t full[2], barA, barB;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) tmem_alloc(&tmem_sh, 256);
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&barA, 1);
    mbar_init(&barB, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // factor tables, and zeros in the stage-B operands (kl = 17..31 stay zero)
  for (int i = tid; i < kTabBytes4 / 16; i += kThreads4)
    reinterpret_cast<uint4*>(sm + kOffFac)[i] = __ldg(reinterpret_cast<const uint4*>(tabs) + i);
  for (int i = tid; i < 2 * kOpB / 16; i += kThreads4)
    reinterpret_cast<uint4*>(sm + kOffOpB)[i] = make_uint4(0u, 0u, 0u, 0u);
  // this thread's twiddles W1024^(xl kl) / 2, xl = lane
  float2 twr[17];
#pragma unroll
  for (int kl = 0; kl < 17; ++kl) twr[kl] = __ldg(tw + lane * 17 + kl);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t sbase = smem_u32(sm);
  constexpr uint32_t idA = make_idesc(128, kNA) | (1u << 15);  // A MN-major
  constexpr uint32_t idB = make_idesc(128, kNB) | (1u << 15);
  uint32_t phA = 0, phB = 0;
  // thread 0: copies issued into buffer b and not yet waited for, and the
  // number of completed waits on full[b] (its next parity)
  int issued[2] = {0, 0};
  uint32_t used[2] = {0u, 0u};

  if (tid == 0 && (int)blockIdx.x < ntasks) {
    const int t = blockIdx.x, g = t % n_groups, y = y0 + t / n_groups;
    mbar_arrive_tx(&full[0], (uint32_t)kTile);
    tma_load_3d(sm + kOffTile, &tm, 0, y * 32, g * kPx, &full[0]);
    issued[0] = 1;
  }
  int it = 0;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x, ++it) {
    const int s = it & 1;
    const int g = t % n_groups, y = y0 + t / n_groups;
    if (tid == 0) {
      // the next task's tile goes into the other buffer, whose stage-A MMAs
      // (previous task) have completed
      const int tn = t + (int)gridDim.x;
      if (tn < ntasks) {
        const int gn = tn % n_groups, yn = y0 + tn / n_groups;
        mbar_arrive_tx(&full[s ^ 1], (uint32_t)kTile);
        tma_load_3d(sm + kOffTile + (s ^ 1) * kTile, &tm, 0, yn * 32, gn * kPx, &full[s ^ 1]);
        issued[s ^ 1] = 1;
      }
      const bool ok = mbar_wait(&full[s], used[s] & 1u);
      if (!ok) {
        abort_sh = 1;
        st_or(st, EER4D_ST_TIMEOUT);
      } else {
        issued[s] = 0;
        ++used[s];
        tc_fence_after();
        const uint32_t tile = sbase + kOffTile + s * kTile;
        const uint32_t fa_hi = sbase + kOffFac, fa_lo = fa_hi + kFacA;
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t a = desc_mn_sw64(tile + mb * 4 * 2048 + ks * 1024, 2048, 512);
            mma_f16(tmem + colA(mb), a, desc_kmajor(fa_hi + ks * 256, 128, 512), idA, ks > 0);
            mma_f16(tmem + colA(mb), a, desc_kmajor(fa_lo + ks * 256, 128, 512), idA, 1u);
          }
        mma_commit(&barA);
      }
    }
    __syncthreads();
    if (abort_sh) break;
    if (!mbar_wait(&barA, phA)) {
      abort_sh = 1;
      st_or(st, EER4D_ST_TIMEOUT);
    }
    phA ^= 1u;
    __syncthreads();
    if (abort_sh) break;
    tc_fence_after();
    // ---- epilogue A: twiddle, halve, split into the stage-B operand -------
#pragma unroll 1
    for (int mb = 0; mb < 2; ++mb) {
      const int b = 4 * mb + warp;  // pixel of this warp's 32 rows (xl = lane)
      float v[48];
      {
        float a[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + colA(mb), a);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = a[i];
        float c[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + colA(mb) + 32u, c);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[32 + i] = c[i];
      }
      float dr[24], di[24];
#pragma unroll
      for (int kl = 0; kl < 24; ++kl) {
        if (kl < 17) {
          const float2 w = twr[kl];
          dr[kl] = v[2 * kl] * w.x - v[2 * kl + 1] * w.y;
          di[kl] = v[2 * kl] * w.y + v[2 * kl + 1] * w.x;
        } else {
          dr[kl] = di[kl] = 0.f;
        }
      }
      unsigned char* ob = sm + kOffOpB + b * 4096;
#pragma unroll
      for (int part = 0; part < 2; ++part) {        // 0: real parts (row xl), 1: imaginary (32 + xl)
        const uint32_t row = (uint32_t)(part * 32 + lane);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {            // kl = 8 ch .. 8 ch + 7
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int k0 = 8 * ch + 2 * q;
            const float x0 = part ? di[k0] : dr[k0], x1 = part ? di[k0 + 1] : dr[k0 + 1];
            const __half2 h = __floats2half2_rn(x0, x1);
            const float2 hf = __half22float2(h);
            hi[q] = *reinterpret_cast<const uint32_t*>(&h);
            lo[q] = pack_h2(x0 - hf.x, x1 - hf.y);
          }
          const uint32_t o = sw64_chunk(row, (uint32_t)ch);
          *reinterpret_cast<uint4*>(ob + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(ob + kOpB + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- stage B ----------------------------------------------------------
    if (tid == 0) {
      tc_fence_after();
      const uint32_t oh = sbase + kOffOpB, ol = oh + kOpB;
      const uint32_t fb_hi = sbase + kOffFac + 2 * kFacA, fb_lo = fb_hi + kFacB;
#pragma unroll
      for (int mb = 0; mb < 2; ++mb)
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t ah = desc_mn_sw64(oh + mb * 4 * 4096 + ks * 1024, 4096, 512);
          const uint64_t al = desc_mn_sw64(ol + mb * 4 * 4096 + ks * 1024, 4096, 512);
          const uint64_t bh = desc_kmajor(fb_hi + ks * 256, 128, 1024);
          const uint64_t bl = desc_kmajor(fb_lo + ks * 256, 128, 1024);
          const uint32_t d = tmem + colB(mb);
          mma_f16(d, ah, bh, idB, ks > 0);
          mma_f16(d, al, bh, idB, 1u);
          mma_f16(d, ah, bl, idB, 1u);
        }
      mma_commit(&barB);
    }
    if (!mbar_wait(&barB, phB)) {
      abort_sh = 1;
      st_or(st, EER4D_ST_TIMEOUT);
    }
    phB ^= 1u;
    __syncthreads();
    if (abort_sh) break;
    tc_fence_after();
    // ---- epilogue B: X(k) of 8 pixels into the staging rows [k][b] --------
    float2* stg = reinterpret_cast<float2*>(sm + kOffOut);
#pragma unroll 1
    for (int mb = 0; mb < 2; ++mb) {
      const int b = 4 * mb + warp, kl = lane;  // this warp's rows: (pixel b, kl = lane)
      float o[64];
      {
        float a[32];
        const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + colB(mb);
        tmem_ld32(ta, a);
#pragma unroll
        for (int i = 0; i < 32; ++i) o[i] = a[i];
        tmem_ld32(ta + 32, a);
#pragma unroll
        for (int i = 0; i < 32; ++i) o[32 + i] = a[i];
      }
      if (kl <= 16) {
#pragma unroll
        for (int kh = 0; kh < 32; ++kh) {
          const float2 xv = make_float2(2.f * o[2 * kh], 2.f * o[2 * kh + 1]);
          const int k = kl + 32 * kh;
          if (k <= 512) {
            if (kl == 0 || kh < 16) stg[k * kOutPitch + b] = xv;
          } else if (kl >= 1 && kl <= 15 && kh >= 16) {
            stg[(1024 - k) * kOutPitch + b] = make_float2(xv.x, -xv.y);  // X(1024 - k) = conj X(k)
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    // ---- staged rows out: X1[k][y][p0 .. p0 + 7], 16 bytes per thread -----
    float2* dst = X1 + (size_t)y * P_pad + (size_t)g * kPx;
    const bool rows_ok = EER4D_IN_RANGE(y, Ny, st) && EER4D_IN_RANGE(g * kPx + kPx - 1, P_pad, st);
    for (int i = tid; rows_ok && i < kNk * (kPx / 2); i += kThreads4) {
      const int k = i >> 2, q = i & 3;
      const float2 a = stg[k * kOutPitch + 2 * q], c = stg[k * kOutPitch + 2 * q + 1];
      *reinterpret_cast<float4*>(dst + (size_t)k * Ny * P_pad + 2 * q) = make_float4(a.x, a.y, c.x, c.y);
    }
  }
  // a copy still in flight after an abort lands in this CTA's shared memory:
  // wait for it (bounded) before the CTA exits
  if (tid == 0) {
    for (int b = 0; b < 2; ++b)
      if (issued[b]) mbar_wait(&full[b], used[b] & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

}  // namespace

static __half neg_h(__half h) { return __ushort_as_half((unsigned short)(__half_as_ushort(h) ^ 0x8000u)); }

// Host: factor tables (hi, lo of the stage-A and stage-B matrices in their
// shared-memory layouts) and the twiddles W1024^(xl kl) / 2.
cudaError_t make_dftx_tc4(eer4d_plan* p) {
  std::vector<unsigned char> tab(kTabBytes4, 0);
  auto put = [&](int base, int n, int k, int K, __half v) {
    *reinterpret_cast<__half*>(tab.data() + base + fac_off(n, k, K)) = v;
  };
  // stage A: n = 2 kl + c, k = xh: (cos, -sin)(2 pi xh kl / 32)
  for (int kl = 0; kl < 17; ++kl)
    for (int c = 0; c < 2; ++c)
      for (int xh = 0; xh < 32; ++xh) {
        __half hi, lo;
        dft_split_factor(32, kl, xh, c, &hi, &lo);
        put(0, 2 * kl + c, xh, 32, hi);
        put(kFacA, 2 * kl + c, xh, 32, lo);
      }
  // stage B: n = 2 kh + c; k < 32: coefficient of Re D(xl = k), k >= 32: of
  // Im D(xl = k - 32).  Out = D W: re = Dr Wr - Di Wi, im = Dr Wi + Di Wr.
  for (int kh = 0; kh < 32; ++kh)
    for (int xl = 0; xl < 32; ++xl) {
      __half rh, rl, ih, il;  // Wr, Wi = (cos, -sin)(2 pi xl kh / 32)
      dft_split_factor(32, kh, xl, 0, &rh, &rl);
      dft_split_factor(32, kh, xl, 1, &ih, &il);
      const int b0 = 2 * kFacA;
      put(b0, 2 * kh, xl, 64, rh);
      put(b0, 2 * kh, 32 + xl, 64, neg_h(ih));
      put(b0, 2 * kh + 1, xl, 64, ih);
      put(b0, 2 * kh + 1, 32 + xl, 64, rh);
      put(b0 + kFacB, 2 * kh, xl, 64, rl);
      put(b0 + kFacB, 2 * kh, 32 + xl, 64, neg_h(il));
      put(b0 + kFacB, 2 * kh + 1, xl, 64, il);
      put(b0 + kFacB, 2 * kh + 1, 32 + xl, 64, rl);
    }
  std::vector<float2> tw(32 * 17);
  const double tp = 6.283185307179586476925286766559;
  for (int xl = 0; xl < 32; ++xl)
    for (int kl = 0; kl < 17; ++kl) {
      const long long e = ((long long)xl * kl) % 1024;
      tw[xl * 17 + kl] = make_float2((float)(0.5 * cos(tp * (double)e / 1024.0)),
                                     (float)(-0.5 * sin(tp * (double)e / 1024.0)));
    }
  cudaError_t e = cudaMalloc(&p->d_tc4_tabs, tab.size());
  if (e != cudaSuccess) return e;
  if ((e = cudaMemcpy(p->d_tc4_tabs, tab.data(), tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if ((e = cudaMalloc(&p->d_tc4_tw, sizeof(float2) * tw.size())) != cudaSuccess) return e;
  return cudaMemcpy(p->d_tc4_tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
}

bool dftx_tc4_ok(const eer4d_plan* p) {
  return p->g.scan_nx == 1024 && p->P_pad % kPx == 0 && p->cstride % 8 == 0 && p->d_tc4_tabs &&
         encode_fn() != nullptr;
}

// X1[k][y][p] for the scan rows [y0, y1): one task per (row, 8-pixel group).
cudaError_t launch_stage1_tc4(const eer4d_plan* p, const __half* counts, float2* X1, int y0, int y1,
                              uint32_t* st, cudaStream_t s) {
  if (y1 <= y0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(counts) & 15) != 0) return cudaErrorInvalidValue;
  const long long NR = (long long)p->g.scan_ny * 1024;
  CUtensorMap map;
  const cuuint64_t gdim[3] = {32, (cuuint64_t)(NR / 32), (cuuint64_t)p->P_pad};
  const cuuint64_t gstride[2] = {64, (cuuint64_t)p->cstride * 2};
  const cuuint32_t box[3] = {32, 32, (cuuint32_t)kPx};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<__half*>(counts), gdim,
                  gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)kSmem4 + 1024;
  cudaError_t e = ensure_smem((const void*)k_dftx_tc4, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int n_groups = p->P_pad / kPx;
  const long long ntasks = (long long)n_groups * (y1 - y0);
  if (ntasks >= (1ll << 31)) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(ntasks, nsm);
  stage_begin(p, EER4D_STAGE_DFT_X, s);
  k_dftx_tc4<<<grid, kThreads4, smem, s>>>(map, p->d_tc4_tabs, p->d_tc4_tw, X1, n_groups,
                                           (int)p->g.scan_ny, p->P_pad, y0, (int)ntasks, st);
  count_launches(1);
  stage_end(p, EER4D_STAGE_DFT_X, s);
  return cudaGetLastError();
}
