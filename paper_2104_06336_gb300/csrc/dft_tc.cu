// Split-FP16 tensor-core DFT along the scan x axis (the G function of Sec. IV,
// first of its two 1D transforms) on the 5th-generation tensor cores.
//
// X1[p, y][k] = sum_x counts[p, y][x] exp(-2 pi i k x / Nx), k = 0 .. Nx/2,
// is a real GEMM D = A B^T with A[m][x] = counts (pixel rows at one scan row
// y; integers <= 2048, exact in fp16) and B[n][x] = (cos, -sin)(2 pi k x/Nx)
// for n = 2k, 2k+1.  B = B_hi + B_lo with B_hi = fp16(B), B_lo = fp16(B - B_hi)
// (about 22 significant bits together); both products accumulate in one FP32
// accumulator in tensor memory: D = A B_hi^T + A B_lo^T.
//
// Per CTA: 128 pixel rows (M) at one y; N tiles of 256 columns; K tiles of 64.
// Operands are staged in shared memory in the no-swizzle K-major core-matrix
// layout (8 rows x 16 bytes per core matrix; leading-dimension offset 128 B
// between K-adjacent core matrices, stride offset 1024 B between 8-row
// groups).  One thread issues tcgen05.mma (kind::f16, M = 128, N = 256,
// K = 16) and commits to an mbarrier; every wait on it is bounded by a
// %globaltimer limit and, on expiry, sets EER4D_ST_TIMEOUT, stops issuing and
// still frees the tensor memory.
#include <cuda.h>
#include <math.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kM = 128;       // rows per CTA (pixels)
constexpr int kN = 256;       // accumulator columns per N tile
constexpr int kK = 64;        // K per stage (fp16: 128 bytes per row)
constexpr int kThreadsTC = 256;
constexpr int kTileA = kM * kK * 2;   // 16 KB
constexpr int kTileB = kN * kK * 2;   // 32 KB

// counts: fp16 [P_pad][Ny*Nx]; Bhi/Blo: tile-blocked [NT][KT][kN x kK] in the
// shared core-matrix layout; X1: complex64 [nkx][Ny][P_pad].  grid = (pixel
// tiles of 128, scan rows y1 - y0).  vec: counts rows 16-byte aligned.
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_dftx_tc(const __half* __restrict__ counts, const uint4* __restrict__ Bhi,
              const uint4* __restrict__ Blo, float2* __restrict__ X1, int Nx, int KT, int NT,
              int nkx, int P_pad, int Ny, long long NR, int y0, int vec, uint32_t* st) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* sA = sm;
  unsigned char* sBh = sm + kTileA;
  unsigned char* sBl = sm + kTileA + kTileB;
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int p0 = blockIdx.x * kM;
  const int y = y0 + blockIdx.y;

  if (warp == 0) tmem_alloc(&tmem_sh, kN);
  if (tid == 0) {
    mbar_init(&mbar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  constexpr uint32_t idesc = make_idesc(kM, kN);
  uint32_t phase = 0;

  for (int nt = 0; nt < NT && !abort_sh; ++nt) {
    for (int kt = 0; kt < KT; ++kt) {
      // A tile: rows p0..p0+127, x = kt*64 .. +63 (zero outside the data)
      for (int c = tid; c < kM * (kK / 8); c += kThreadsTC) {
        const int r = c >> 3, kc = c & 7;
        const int p = p0 + r, x = kt * kK + kc * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (p < P_pad) {
          const __half* src = counts + (size_t)p * NR + (size_t)y * Nx + x;
          if (vec && x + 8 <= Nx) {
            v = __ldg(reinterpret_cast<const uint4*>(src));
          } else {
            __half h[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) h[i] = (x + i < Nx) ? src[i] : __float2half(0.f);
            v = *reinterpret_cast<const uint4*>(h);
          }
        }
        *reinterpret_cast<uint4*>(sA + cm_off(r, kc * 8)) = v;
      }
      // B tiles: contiguous pre-arranged blocks
      const size_t tb = ((size_t)nt * KT + kt) * (kTileB / 16);
      for (int c = tid; c < kTileB / 16; c += kThreadsTC) {
        reinterpret_cast<uint4*>(sBh)[c] = __ldg(Bhi + tb + c);
        reinterpret_cast<uint4*>(sBl)[c] = __ldg(Blo + tb + c);
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA), bh0 = smem_u32(sBh), bl0 = smem_u32(sBl);
#pragma unroll
        for (int ks = 0; ks < kK / 16; ++ks) {
          const uint64_t ad = make_desc(a0 + ks * 256);
          mma_f16(tmem, ad, make_desc(bh0 + ks * 256), idesc, (kt | ks) != 0);
          mma_f16(tmem, ad, make_desc(bl0 + ks * 256), idesc, 1u);
        }
        mma_commit(&mbar);
      }
      // the MMAs read the staged tiles: wait before they are overwritten
      const bool ok = mbar_wait(&mbar, phase);
      phase ^= 1u;
      if (!ok) {
        if (tid == 0) abort_sh = 1;
        st_or(st, EER4D_ST_TIMEOUT);
      }
      __syncthreads();
      if (abort_sh) break;
    }
    if (abort_sh) break;
    // epilogue: accumulator columns -> X1 (column 2j re, 2j+1 im of k = nt*128 + j)
    tc_fence_after();
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    const int p = p0 + row;
#pragma unroll 1
    for (int j = 0; j < (kN / 2) / 16; ++j) {
      const int col = half * (kN / 2) + j * 16;
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col, v);
      if (p < P_pad) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = nt * (kN / 2) + (col >> 1) + i;
          if (k < nkx) X1[((size_t)k * Ny + y) * P_pad + p] = make_float2(v[2 * i], v[2 * i + 1]);
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (abort_sh) mbar_wait(&mbar, phase ^ 1u);  // bounded: let an in-flight MMA retire
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kN);
  }
}

// ---------------------------------------------------------------------------
// Pipelined form (TMA -> 2-stage shared ring -> tcgen05.mma -> double-buffered
// TMEM accumulators -> epilogue warps), used when the TMA alignment rules hold
// (Nx % 8 == 0, 16-byte aligned counts).  Warp 0 lane 0 is the producer: the
// A tile (128 pixel rows x 64 frames of fp16 counts) by a 2D tensor-map load
// with 128-byte swizzle, the pre-tiled B_hi / B_lo tiles by 1D bulk copies, all
// completing on full[s].  Warp 1 lane 0 issues the MMAs and commits empty[s]
// (stage free) and, per N tile, accf[b] (accumulator b ready).  Warps 4..7
// drain accumulator b to X1 and arrive on acce[b].  Every wait is bounded.
constexpr int kStages = 2;
constexpr int kStageBytes = kTileA + 2 * kTileB;  // 80 KB, a multiple of 1024

__global__ void __launch_bounds__(kThreadsTC, 1)
    k_dftx_tc2(const __grid_constant__ CUtensorMap tmA, const unsigned char* __restrict__ Bhi,
               const unsigned char* __restrict__ Blo, float2* __restrict__ X1, int Nx, int KT,
               int NT, int nlast, int nkx, int P_pad, int Ny, int y0, uint32_t* st) {
  extern __shared__ unsigned char sm_raw[];
  const uint32_t raw = smem_u32(sm_raw);
  unsigned char* sm = sm_raw + (((raw + 1023u) & ~1023u) - raw);  // 1024-aligned stages
  __shared__ uint64_t full[kStages], empty[kStages], accf[2], acce[2];
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int abort_sh;
  __shared__ int wflag[kThreadsTC / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int p0 = blockIdx.x * kM;
  const int y = y0 + blockIdx.y;
  if (warp == 2) tmem_alloc(&tmem_sh, 2 * kN);
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 4);
    }
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t idesc_full = make_idesc(kM, kN), idesc_last = make_idesc(kM, nlast);
  const int total = NT * KT;

  if (warp == 0 && lane == 0) {  // ---- producer
    for (int it = 0; it < total && !abort_sh; ++it) {
      const int s = it % kStages, k = it / kStages;
      if (it >= kStages && !mbar_wait(&empty[s], (k - 1) & 1)) {
        abort_sh = 1;
        st_or(st, EER4D_ST_TIMEOUT);
        break;
      }
      const int nt = it / KT, kt = it - nt * KT;
      unsigned char* sa = sm + s * kStageBytes;
      // the last N tile holds only nlast rows (a multiple of 16 = two 8-row groups)
      const uint32_t bbytes = (uint32_t)((nt == NT - 1 ? nlast : kN) * kK * 2);
      mbar_arrive_tx(&full[s], (uint32_t)kTileA + 2u * bbytes);
      tma_load_2d(sa, &tmA, y * Nx + kt * kK, p0, &full[s]);
      const size_t tb = ((size_t)nt * KT + kt) * kTileB;
      bulk_load(sa + kTileA, Bhi + tb, bbytes, &full[s]);
      bulk_load(sa + kTileA + kTileB, Blo + tb, bbytes, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {  // ---- MMA issuer
    int it = 0;
    for (int nt = 0; nt < NT && !abort_sh; ++nt) {
      const int b = nt & 1, u = nt >> 1;
      if (nt >= 2 && !mbar_wait(&acce[b], (u - 1) & 1)) {
        abort_sh = 1;
        st_or(st, EER4D_ST_TIMEOUT);
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(b * kN);
      for (int kt = 0; kt < KT; ++kt, ++it) {
        const int s = it % kStages, k = it / kStages;
        if (!mbar_wait(&full[s], k & 1)) {
          abort_sh = 1;
          st_or(st, EER4D_ST_TIMEOUT);
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(sm + s * kStageBytes);
        const uint32_t idesc = nt == NT - 1 ? idesc_last : idesc_full;
#pragma unroll
        for (int ks = 0; ks < kK / 16; ++ks) {
          const uint64_t ad = make_desc_sw128(sa + ks * 32);
          mma_f16(d, ad, make_desc(sa + kTileA + ks * 256), idesc, (kt | ks) != 0);
          mma_f16(d, ad, make_desc(sa + kTileA + kTileB + ks * 256), idesc, 1u);
        }
        mma_commit(&empty[s]);
      }
      if (abort_sh) break;
      mma_commit(&accf[b]);
    }
  } else if (warp >= 4) {  // ---- epilogue
    const int quarter = warp & 3;
    const int p = p0 + quarter * 32 + lane;
    for (int nt = 0; nt < NT; ++nt) {
      const int b = nt & 1, u = nt >> 1;
      if (lane == 0) {
        const bool ok = !abort_sh && mbar_wait(&accf[b], u & 1);
        if (!ok && !abort_sh) {
          abort_sh = 1;
          st_or(st, EER4D_ST_TIMEOUT);
        }
        wflag[warp] = ok;
      }
      __syncwarp();
      if (!wflag[warp]) break;
      tc_fence_after();
      const uint32_t tb = tmem + (uint32_t)(b * kN) + ((uint32_t)(quarter * 32) << 16);
      const int ncols = nt == NT - 1 ? nlast : kN;
#pragma unroll 1
      for (int j = 0; j < ncols / 16; ++j) {
        float v[16];
        tmem_ld16(tb + (uint32_t)(j * 16), v);
        if (p < P_pad) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int k = nt * (kN / 2) + j * 8 + i;
            if (k < nkx) X1[((size_t)k * Ny + y) * P_pad + p] = make_float2(v[2 * i], v[2 * i + 1]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
  }
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * kN);
  }
}

}  // namespace

// Host: one DFT factor exp(-2 pi i k x / n), component c (0 = cos, 1 = -sin),
// from the exact integer phase index (k x) mod n in double, split as
// hi = fp16(w), lo = fp16(w - hi).
void dft_split_factor(int n, long long k, long long x, int c, __half* hi, __half* lo) {
  const double tp = 6.283185307179586476925286766559;
  const long long e = (k * x) % n;
  const double w = c ? -sin(tp * (double)e / n) : cos(tp * (double)e / n);
  *hi = __float2half_rn((float)w);
  *lo = __float2half_rn((float)(w - (double)__half2float(*hi)));
}

extern "C" int eer4d_dft_split_factors(int n, int n_k, uint16_t* h_hi, uint16_t* h_lo) {
  if (n < 1 || n > 65536 || n_k < 1 || n_k > n || !h_hi || !h_lo) return EER4D_EINVAL;
  for (int k = 0; k < n_k; ++k)
    for (int x = 0; x < n; ++x)
      for (int c = 0; c < 2; ++c) {
        __half hi, lo;
        dft_split_factor(n, k, x, c, &hi, &lo);
        const size_t o = ((size_t)k * n + x) * 2 + c;
        h_hi[o] = __half_as_ushort(hi);
        h_lo[o] = __half_as_ushort(lo);
      }
  return EER4D_OK;
}

// Host: the tile-blocked split DFT matrix for this plan's Nx.
cudaError_t make_dftx_tc(eer4d_plan* p) {
  const int Nx = p->g.scan_nx, nkx = p->nkx;
  const int KT = (Nx + kK - 1) / kK;
  const int NT = (2 * nkx + kN - 1) / kN;
  const size_t tile_elems = (size_t)kN * kK;
  std::vector<__half> hi((size_t)NT * KT * tile_elems), lo(hi.size());
  for (int nt = 0; nt < NT; ++nt)
    for (int kt = 0; kt < KT; ++kt) {
      __half* th = hi.data() + ((size_t)nt * KT + kt) * tile_elems;
      __half* tl = lo.data() + ((size_t)nt * KT + kt) * tile_elems;
      for (int r = 0; r < kN; ++r)
        for (int k = 0; k < kK; ++k) {
          const int n = nt * kN + r, x = kt * kK + k, kx = n >> 1;
          __half h = __float2half_rn(0.f), l = h;
          if (x < Nx && kx < nkx) dft_split_factor(Nx, kx, x, n & 1, &h, &l);
          const size_t o = ((size_t)(r >> 3) * 1024 + (size_t)(k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2) / 2;
          th[o] = h;
          tl[o] = l;
        }
    }
  cudaError_t e = cudaMalloc(&p->d_dft_hi, hi.size() * sizeof(__half));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&p->d_dft_lo, lo.size() * sizeof(__half));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(p->d_dft_hi, hi.data(), hi.size() * sizeof(__half), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(p->d_dft_lo, lo.data(), lo.size() * sizeof(__half), cudaMemcpyHostToDevice);
}

cudaError_t launch_stage1_tc(const eer4d_plan* p, const __half* counts, float2* X1, int y0, int y1,
                             uint32_t* st, cudaStream_t s) {
  if (y1 <= y0) return cudaSuccess;
  // 1024 columns: the four-step form (two DFT-32 contractions per row)
  if (dftx_tc4_ok(p) && (reinterpret_cast<uintptr_t>(counts) & 15) == 0)
    return launch_stage1_tc4(p, counts, X1, y0, y1, st, s);
  const int Nx = p->g.scan_nx, Ny = p->g.scan_ny;
  const int KT = (Nx + kK - 1) / kK;
  const int NT = (2 * p->nkx + kN - 1) / kN;
  const long long NR = (long long)Ny * Nx;
  const long long CS = p->cstride;  // counts row stride
  // pipelined TMA form when its alignment rules hold: x coordinates (frames)
  // at multiples of 8 fp16 (16 bytes), row stride CS*2 a multiple of 16
  EncodeTiledFn enc = encode_fn();
  if (enc && Nx % 8 == 0 && CS % 8 == 0 && (reinterpret_cast<uintptr_t>(counts) & 15) == 0) {
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)NR, (cuuint64_t)p->P_pad};
    const cuuint64_t gstride[1] = {(cuuint64_t)CS * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kK, (cuuint32_t)kM};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half*>(counts), gdim, gstride,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
      const size_t smem = (size_t)kStages * kStageBytes + 1024;
      cudaError_t e = ensure_smem((const void*)k_dftx_tc2, smem);
      if (e != cudaSuccess) return e;
      dim3 grid((p->P_pad + kM - 1) / kM, y1 - y0);
      stage_begin(p, EER4D_STAGE_DFT_X, s);
      const int rem = 2 * p->nkx - (NT - 1) * kN;  // columns of the last N tile
      const int nlast = (rem + 15) / 16 * 16;
      k_dftx_tc2<<<grid, kThreadsTC, smem, s>>>(
          map, reinterpret_cast<const unsigned char*>(p->d_dft_hi),
          reinterpret_cast<const unsigned char*>(p->d_dft_lo), X1, Nx, KT, NT, nlast, p->nkx,
          p->P_pad, Ny, y0, st);
      count_launches(1);
      stage_end(p, EER4D_STAGE_DFT_X, s);
      return cudaGetLastError();
    }
  }
  const int vec = (Nx % 8 == 0) && (CS % 8 == 0);
  const size_t smem = kTileA + 2 * kTileB;
  cudaError_t e = ensure_smem((const void*)k_dftx_tc, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((p->P_pad + kM - 1) / kM, y1 - y0);
  stage_begin(p, EER4D_STAGE_DFT_X, s);
  k_dftx_tc<<<grid, kThreadsTC, smem, s>>>(counts, reinterpret_cast<const uint4*>(p->d_dft_hi),
                                           reinterpret_cast<const uint4*>(p->d_dft_lo), X1, Nx, KT,
                                           NT, p->nkx, p->P_pad, Ny, CS, y0, vec, st);
  count_launches(1);
  stage_end(p, EER4D_STAGE_DFT_X, s);
  return cudaGetLastError();
}
