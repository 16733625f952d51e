// Register-resident four-step FFT for power-of-two lengths N = R1 * R2
// (R1 >= R2, both in {4, 8, 16, 32}): the two large scan-axis transforms of
// the G function (Sec. IV) at the sizes of the paper's scans.
//
// With n = R2 j1 + j2 and k = k1 + R1 k2:
//   X(k1 + R1 k2) = sum_j2 W_R2^{j2 k2} W_N^{j2 k1} [sum_j1 W_R1^{j1 k1} x(R2 j1 + j2)].
// Pass 1: one thread per (j2, transform) loads its R1 strided inputs straight
// from global memory into registers (R1 independent loads in flight), does the
// R1-point DFT in registers, applies the twiddle W_N^{j2 k1} (exact integer
// index into the plan's table) and stores to shared memory.  Pass 2: one
// thread per (k1, transform) reads R2 values and does the R2-point DFT.
// Shared rows are padded to R2 + 1 entries so the strided pass-2 reads hit
// distinct banks.
#pragma once

#include "common.cuh"

// exp(-2 pi i m / 32) for m = 0..15 (values of cos/sin at multiples of pi/16)
__device__ __forceinline__ float2 w32(int m) {
  switch (m) {
    case 0: return make_float2(1.0f, 0.0f);
    case 1: return make_float2(0.9807852506637573f, -0.19509032368659973f);
    case 2: return make_float2(0.9238795042037964f, -0.3826834261417389f);
    case 3: return make_float2(0.8314695954322815f, -0.5555702447891235f);
    case 4: return make_float2(0.7071067690849304f, -0.7071067690849304f);
    case 5: return make_float2(0.5555702447891235f, -0.8314695954322815f);
    case 6: return make_float2(0.3826834261417389f, -0.9238795042037964f);
    case 7: return make_float2(0.19509032368659973f, -0.9807852506637573f);
    case 8: return make_float2(0.0f, -1.0f);
    case 9: return make_float2(-0.19509032368659973f, -0.9807852506637573f);
    case 10: return make_float2(-0.3826834261417389f, -0.9238795042037964f);
    case 11: return make_float2(-0.5555702447891235f, -0.8314695954322815f);
    case 12: return make_float2(-0.7071067690849304f, -0.7071067690849304f);
    case 13: return make_float2(-0.8314695954322815f, -0.5555702447891235f);
    case 14: return make_float2(-0.9238795042037964f, -0.3826834261417389f);
    default: return make_float2(-0.9807852506637573f, -0.19509032368659973f);
  }
}

__host__ __device__ constexpr int bitrev_c(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int log2_c(int n) { return n <= 1 ? 0 : 1 + log2_c(n / 2); }

// In-register R-point DFT (R a power of two <= 32), natural order in and out:
// radix-2 decimation in frequency, then the bit-reversal permutation (free
// register renaming once unrolled).  DIR = +1 forward, -1 inverse (unscaled).
template <int R, int DIR>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
#pragma unroll
  for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int blk = 0; blk < R; blk += 2 * span) {
#pragma unroll
      for (int j = 0; j < span; ++j) {
        const float2 a = v[blk + j], b = v[blk + j + span];
        v[blk + j] = make_float2(a.x + b.x, a.y + b.y);
        const float2 d = make_float2(a.x - b.x, a.y - b.y);
        if (j == 0) {
          v[blk + j + span] = d;
        } else {
          float2 w = w32(j * (32 / (2 * span)));
          if (DIR < 0) w.y = -w.y;
          v[blk + j + span] = make_float2(d.x * w.x - d.y * w.y, d.x * w.y + d.y * w.x);
        }
      }
    }
  }
  constexpr int B = log2_c(R);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = bitrev_c(i, B);
    if (r > i) {
      const float2 t = v[i];
      v[i] = v[r];
      v[r] = t;
    }
  }
}

__device__ __forceinline__ float2 twid_dir(const float2* __restrict__ tw, int e, int dir) {
  float2 w = __ldg(tw + e);
  if (dir < 0) w.y = -w.y;
  return w;
}

// Column transforms of a [N][ld] complex array (element n of column c at
// n*ld_in + c), CB columns per CTA, batch = blockIdx.y.  Output element n of
// column c goes to n*ld_out + c, or with TOUT (transposed output) to
// c*ld_out + n, so each column's spectrum is contiguous.  In place is allowed
// only without TOUT (every input of the CTA is read before the barrier, every
// output written after it, and CTAs own disjoint columns).
template <int R1, int R2, int CB, int DIR, bool TOUT>
__device__ __forceinline__ int colfft_yidx(int k1, int col, int j2) {
  return TOUT ? ((col * R1 + k1) * (R2 + 1) + 2 * col + j2) : ((k1 * CB + col) * (R2 + 1) + j2);
}

template <int R1, int R2, int CB, int DIR, bool TOUT>
__global__ void __launch_bounds__((R1 > R2 ? R1 : R2) * CB)
    k_colfft_reg(const float2* in, float2* out, const float2* __restrict__ tw, int ncols, int ld_in,
                 int ld_out, long long bs_in, long long bs_out, float scale) {
  constexpr int NT = (R1 > R2 ? R1 : R2) * CB;
  extern __shared__ float2 sm[];
  const int c0 = blockIdx.x * CB;
  in += blockIdx.y * bs_in;
  out += blockIdx.y * bs_out;
  for (int g = threadIdx.x; g < R2 * CB; g += NT) {
    const int col = g % CB, j2 = g / CB, c = c0 + col;
    float2 v[R1];
#pragma unroll
    for (int j1 = 0; j1 < R1; ++j1)
      v[j1] = c < ncols ? in[(size_t)(R2 * j1 + j2) * ld_in + c] : make_float2(0.f, 0.f);
    dft_reg<R1, DIR>(v);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const float2 t = (k1 == 0) ? v[k1] : cmul(v[k1], twid_dir(tw, j2 * k1, DIR));
      sm[colfft_yidx<R1, R2, CB, DIR, TOUT>(k1, col, j2)] = t;
    }
  }
  __syncthreads();
  for (int g = threadIdx.x; g < R1 * CB; g += NT) {
    int col, k1;
    if (TOUT) { k1 = g % R1; col = g / R1; } else { col = g % CB; k1 = g / CB; }
    const int c = c0 + col;
    float2 v[R2];
#pragma unroll
    for (int j2 = 0; j2 < R2; ++j2) v[j2] = sm[colfft_yidx<R1, R2, CB, DIR, TOUT>(k1, col, j2)];
    dft_reg<R2, DIR>(v);
    if (c < ncols) {
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int n = k1 + R1 * k2;
        const size_t o = TOUT ? (size_t)c * ld_out + n : (size_t)n * ld_out + c;
        out[o] = make_float2(v[k2].x * scale, v[k2].y * scale);
      }
    }
  }
}

// Real rows (fp16 counts) -> half spectra, scan DFT along x of the G function.
// Row (a, c) = (pixel, scan row y) starts at a*in_sa + c*in_sc; spectrum value
// k goes to k*out_skx + a*out_sa + c*out_sc.  A CTA takes 2*CP consecutive
// pixels at one y and transforms them as CP complex rows z = row_2b + i
// row_2b+1; A(k) = (Z(k) + conj Z(-k))/2, B(k) = -i (Z(k) - conj Z(-k))/2.
// Requires R1 >= R2 so pass 2 has exactly one (k1, b) group per thread.
template <int R1, int R2, int CP>
__global__ void __launch_bounds__(R1 * CP)
    k_rowfft_r2c_reg(const __half* __restrict__ in, float2* out, const float2* __restrict__ tw,
                     int nA, int c0, long long in_sa, long long in_sc, long long out_skx,
                     long long out_sa, long long out_sc) {
  static_assert(R1 >= R2, "R1 >= R2");
  constexpr int N = R1 * R2;
  constexpr int NT = R1 * CP;
  constexpr int PITCH = R2 + 1;
  extern __shared__ float2 sm[];
  const int a0 = blockIdx.x * 2 * CP;
  const int c = c0 + blockIdx.y;
  for (int g = threadIdx.x; g < R2 * CP; g += NT) {
    const int j2 = g % R2, b = g / R2;
    const int ra = a0 + 2 * b, rb = ra + 1;
    const __half* pa = in + ra * in_sa + c * in_sc + j2;
    const __half* pb = in + rb * in_sa + c * in_sc + j2;
    float2 v[R1];
#pragma unroll
    for (int j1 = 0; j1 < R1; ++j1) {
      const float xa = ra < nA ? __half2float(pa[R2 * j1]) : 0.f;
      const float xb = rb < nA ? __half2float(pb[R2 * j1]) : 0.f;
      v[j1] = make_float2(xa, xb);
    }
    dft_reg<R1, 1>(v);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const float2 t = (k1 == 0) ? v[k1] : cmul(v[k1], __ldg(tw + j2 * k1));
      sm[(k1 * CP + b) * PITCH + j2] = t;
    }
  }
  __syncthreads();
  {
    const int b = threadIdx.x % CP, k1 = threadIdx.x / CP;
    float2 v[R2];
#pragma unroll
    for (int j2 = 0; j2 < R2; ++j2) v[j2] = sm[(k1 * CP + b) * PITCH + j2];
    dft_reg<R2, 1>(v);
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) sm[(k1 + R1 * k2) * CP + b] = v[k2];
  }
  __syncthreads();
  constexpr int NK = N / 2 + 1;
  for (int w = threadIdx.x; w < NK * 2 * CP; w += NT) {
    const int i = w % (2 * CP), k = w / (2 * CP);
    const int a = a0 + i;
    if (a >= nA) continue;
    const int b = i >> 1;
    const float2 z = sm[k * CP + b];
    const float2 zm = sm[((N - k) & (N - 1)) * CP + b];
    float2 r;
    if ((i & 1) == 0) r = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    else r = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    out[k * out_skx + a * out_sa + c * out_sc] = r;
  }
}
