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

// Complex sum and difference as packed two-lane fp32 operations (one
// instruction each); a - b is formed as fma(b, -1, a), which rounds once,
// exactly like the scalar subtraction.
__device__ __forceinline__ float2 cadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

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
        v[blk + j] = cadd2(a, b);
        const float2 d = csub2(a, b);
        const int m = j * (32 / (2 * span));  // twiddle exp(-+2 pi i m / 32)
        if (j == 0) {
          v[blk + j + span] = d;
        } else if (m == 8) {  // -i (forward) or +i (inverse): a swap, no products
          v[blk + j + span] = DIR > 0 ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
        } else {
          float2 w = w32(m);
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

// Global-memory access flavours of the tiles below: plain (L1 and L2), or
// STREAM: the intermediate spectrum is read from L2 only (ld.global.cg; it may
// have been written by another CTA of the same launch), the fp16 counts are
// read once (ld.global.cs) and the G function is written once (st.global.cs),
// so the L2 keeps the intermediate.
template <bool STREAM>
__device__ __forceinline__ float2 ld_f2(const float2* p) {
  if (STREAM) return __ldcg(p);
  return *p;
}
template <bool STREAM>
__device__ __forceinline__ void st_f2(float2* p, float2 v) {
  if (STREAM) __stcs(p, v);
  else *p = v;
}
template <bool STREAM>
__device__ __forceinline__ float ld_h(const __half* p) {
  if (STREAM) return __half2float(__ldcs(p));
  return __half2float(*p);
}

// Column transforms of a [N][ld] complex array (element n of column c at
// n*ld_in + c), CB columns per CTA starting at column c0.  Output element n of
// column c goes to n*ld_out + c, or with TOUT (transposed output) to
// c*ld_out + n, so each column's spectrum is contiguous.  In place is allowed
// only without TOUT (every input of the CTA is read before the barrier, every
// output written after it, and CTAs own disjoint columns).  All threads of the
// CTA call it; `sm` holds R1*CB*(R2+1) + 2*CB float2.
template <int R1, int R2, int CB, int DIR, bool TOUT>
__device__ __forceinline__ int colfft_yidx(int k1, int col, int j2) {
  return TOUT ? ((col * R1 + k1) * (R2 + 1) + 2 * col + j2) : ((k1 * CB + col) * (R2 + 1) + j2);
}

template <int R1, int R2, int CB, int DIR, bool TOUT, bool STREAM,
          int NTH = (R1 > R2 ? R1 : R2) * CB>
__device__ __forceinline__ void colfft_tile(const float2* in, float2* out,
                                            const float2* __restrict__ tw4, int c0, int ncols,
                                            int ld_in, int ld_out, float scale, float2* sm) {
  static_assert(R1 == reg_r1(R1 * R2), "twiddle layout of FftDesc::tw4");
  for (int g = threadIdx.x; g < R2 * CB; g += NTH) {
    const int col = g % CB, j2 = g / CB, c = c0 + col;
    float2 v[R1];
#pragma unroll
    for (int j1 = 0; j1 < R1; ++j1)
      v[j1] = c < ncols ? ld_f2<STREAM>(in + (size_t)(R2 * j1 + j2) * ld_in + c)
                        : make_float2(0.f, 0.f);
    dft_reg<R1, DIR>(v);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const float2 t = (k1 == 0) ? v[k1] : cmul(v[k1], twid_dir(tw4, k1 * R2 + j2, DIR));
      sm[colfft_yidx<R1, R2, CB, DIR, TOUT>(k1, col, j2)] = t;
    }
  }
  __syncthreads();
  for (int g = threadIdx.x; g < R1 * CB; g += NTH) {
    int col, k1;
    if (TOUT) { k1 = g % R1; col = g / R1; } else { col = g % CB; k1 = g / CB; }
    const int c = c0 + col;
    float2 v[R2];
#pragma unroll
    for (int j2 = 0; j2 < R2; ++j2) v[j2] = sm[colfft_yidx<R1, R2, CB, DIR, TOUT>(k1, col, j2)];
    dft_reg<R2, DIR>(v);
    if (c < ncols) {
      if (scale != 1.f) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k2] = make_float2(v[k2].x * scale, v[k2].y * scale);
      }
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int n = k1 + R1 * k2;
        const size_t o = TOUT ? (size_t)c * ld_out + n : (size_t)n * ld_out + c;
        st_f2<STREAM>(out + o, v[k2]);
      }
    }
  }
}

// CTA x covers columns [x*CB, x*CB + CB), batch = blockIdx.y.
template <int R1, int R2, int CB, int DIR, bool TOUT>
__global__ void __launch_bounds__((R1 > R2 ? R1 : R2) * CB, 768 / ((R1 > R2 ? R1 : R2) * CB))
    k_colfft_reg(const float2* in, float2* out, const float2* __restrict__ tw4, int ncols, int ld_in,
                 int ld_out, long long bs_in, long long bs_out, float scale) {
  extern __shared__ float2 sm[];
  colfft_tile<R1, R2, CB, DIR, TOUT, false>(in + blockIdx.y * bs_in, out + blockIdx.y * bs_out, tw4,
                                           blockIdx.x * CB, ncols, ld_in, ld_out, scale, sm);
}

// Complex rows of a row-major array (element n of row r at r*ld + n), CB rows
// per CTA from row blockIdx.x * CB, in place: every input of the CTA is read
// in pass 1, before the barrier, and every output written in pass 2, after
// it.  Pass 1 lanes run along j2 (unit stride), pass 2 lanes along k1.  With
// REAL_OUT the real part times scale goes to real_out[r*ld + n] instead.
template <int R1, int R2, int CB, int DIR, bool REAL_OUT>
__global__ void __launch_bounds__((R1 > R2 ? R1 : R2) * CB, 768 / ((R1 > R2 ? R1 : R2) * CB))
    k_rowfft_c2c_reg(float2* data, float* real_out, const float2* __restrict__ tw4, int rows,
                     int ld, float scale) {
  static_assert(R1 == reg_r1(R1 * R2), "twiddle layout of FftDesc::tw4");
  constexpr int NTH = (R1 > R2 ? R1 : R2) * CB;
  constexpr int PITCH = R2 + 1;
  extern __shared__ float2 sm[];
  const int r0 = blockIdx.x * CB;
  for (int g = threadIdx.x; g < R2 * CB; g += NTH) {
    const int b = g / R2, j2 = g % R2, r = r0 + b;
    const float2* src = data + (size_t)r * ld + j2;
    float2 v[R1];
#pragma unroll
    for (int j1 = 0; j1 < R1; ++j1) v[j1] = r < rows ? src[R2 * j1] : make_float2(0.f, 0.f);
    dft_reg<R1, DIR>(v);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1)
      sm[(b * R1 + k1) * PITCH + j2] =
          (k1 == 0) ? v[k1] : cmul(v[k1], twid_dir(tw4, k1 * R2 + j2, DIR));
  }
  __syncthreads();
  for (int g = threadIdx.x; g < R1 * CB; g += NTH) {
    const int b = g / R1, k1 = g % R1, r = r0 + b;
    float2 v[R2];
#pragma unroll
    for (int j2 = 0; j2 < R2; ++j2) v[j2] = sm[(b * R1 + k1) * PITCH + j2];
    dft_reg<R2, DIR>(v);
    if (r >= rows) continue;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const size_t o = (size_t)r * ld + k1 + R1 * k2;
      if (REAL_OUT) real_out[o] = v[k2].x * scale;
      else data[o] = make_float2(v[k2].x * scale, v[k2].y * scale);
    }
  }
}

// Real rows (fp16 counts) -> half spectra, scan DFT along x of the G function.
// Row (a, c) = (pixel, scan row y) starts at a*in_sa + c*in_sc; spectrum value
// k goes to k*out_skx + (a - a_out0)*out_sa + c*out_sc.  The tile takes 2*CP
// consecutive pixels from a0 at scan row c and transforms them as CP complex
// rows z = row_2b + i row_2b+1; A(k) = (Z(k) + conj Z(-k))/2,
// B(k) = -i (Z(k) - conj Z(-k))/2.  Requires R1 >= R2 so pass 2 has exactly
// one (k1, b) group per thread.  `sm` holds max(R1*CP*(R2+1), N*CP) float2.
// FULL: the caller guarantees a0 + 2*CP <= nA (no bounds tests).
template <int R1, int R2, int CP, bool STREAM, bool FULL = false>
__device__ __forceinline__ void rowfft_r2c_tile(const __half* __restrict__ in, float2* out,
                                                const float2* __restrict__ tw4, int nA, int a0,
                                                int a_out0, int c, long long in_sa,
                                                long long in_sc, long long out_skx,
                                                long long out_sa, long long out_sc, float2* sm) {
  static_assert(R1 >= R2, "R1 >= R2");
  static_assert(R1 == reg_r1(R1 * R2), "twiddle layout of FftDesc::tw4");
  constexpr int N = R1 * R2;
  constexpr int NT = R1 * CP;
  constexpr int PITCH = R2 + 1;
  const bool full = FULL || a0 + 2 * CP <= nA;  // every pixel row of the tile exists
  for (int g = threadIdx.x; g < R2 * CP; g += NT) {
    const int j2 = g % R2, b = g / R2;
    const int ra = a0 + 2 * b, rb = ra + 1;
    const __half* pa = in + ra * in_sa + c * in_sc + j2;
    const __half* pb = in + rb * in_sa + c * in_sc + j2;
    float2 v[R1];
    if (full) {
#pragma unroll
      for (int j1 = 0; j1 < R1; ++j1)
        v[j1] = make_float2(ld_h<STREAM>(pa + R2 * j1), ld_h<STREAM>(pb + R2 * j1));
    } else {
#pragma unroll
      for (int j1 = 0; j1 < R1; ++j1) {
        const float xa = ra < nA ? ld_h<STREAM>(pa + R2 * j1) : 0.f;
        const float xb = rb < nA ? ld_h<STREAM>(pb + R2 * j1) : 0.f;
        v[j1] = make_float2(xa, xb);
      }
    }
    dft_reg<R1, 1>(v);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const float2 t = (k1 == 0) ? v[k1] : cmul(v[k1], __ldg(tw4 + k1 * R2 + j2));
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
  // one thread per (k, pair b): both half spectra from Z(k) and Z(-k).  With
  // out_sa == 1 the pair's two values are adjacent and go out as one 16-byte
  // store (callers keep out, out_skx, out_sc and a0 - a_out0 even).
  constexpr int NK = N / 2 + 1;
  for (int w = threadIdx.x; w < NK * CP; w += NT) {
    const int b = w % CP, k = w / CP;
    const int a = a0 + 2 * b;
    if (!FULL && a >= nA) continue;
    const float2 z = sm[k * CP + b];
    const float2 zm = sm[((N - k) & (N - 1)) * CP + b];
    const float2 A = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    const float2 B = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    float2* o = out + k * out_skx + (a - a_out0) * out_sa + c * out_sc;
    if (out_sa == 1 && (FULL || a + 1 < nA)) {
      *reinterpret_cast<float4*>(o) = make_float4(A.x, A.y, B.x, B.y);
    } else {
      o[0] = A;
      if (FULL || a + 1 < nA) o[out_sa] = B;
    }
  }
}

// CTA (x, y) takes pixels [2*CP*x, 2*CP*x + 2*CP) at scan row c0 + y.
template <int R1, int R2, int CP>
__global__ void __launch_bounds__(R1 * CP, 768 / (R1 * CP))
    k_rowfft_r2c_reg(const __half* __restrict__ in, float2* out, const float2* __restrict__ tw4,
                     int nA, int c0, long long in_sa, long long in_sc, long long out_skx,
                     long long out_sa, long long out_sc) {
  extern __shared__ float2 sm[];
  rowfft_r2c_tile<R1, R2, CP, false>(in, out, tw4, nA, blockIdx.x * 2 * CP, 0, c0 + blockIdx.y,
                                     in_sa, in_sc, out_skx, out_sa, out_sc, sm);
}
