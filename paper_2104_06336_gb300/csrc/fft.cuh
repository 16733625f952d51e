// Batched Stockham FFT in shared memory (plain FP32 form of the scan-axis
// transforms; Sec. IV "batched 2D Fast Fourier Transform along the real-space
// coordinates").
//
// A CTA holds nb transforms of length N in two shared buffers (ping-pong).
// Element n of transform b lives at b*sb + n*sn.  Each stage of radix R with
// span Ns does, for butterfly j in [0, N/R):
//   v_r = x[j + r N/R],  v_r *= W_N^{(j mod Ns) r N/(Ns R)},  y = DFT_R(v),
//   out[(j div Ns) Ns R + (j mod Ns) + r Ns] = y_r
// (autosort Stockham; natural order in and out).  Twiddle exponents are exact
// integers < N indexing the table tw[j] = exp(-2 pi i j/N); dir = +1 forward,
// -1 inverse (conjugate twiddles, no scaling).
#pragma once

#include "common.cuh"

__device__ __forceinline__ float2 twid(const float2* __restrict__ tw, int e, int dir) {
  float2 w = __ldg(tw + e);
  return dir > 0 ? w : make_float2(w.x, -w.y);
}

template <int R>
__device__ __forceinline__ void dft_small(float2* v, int dir, const float2* __restrict__ tw, int N);

template <>
__device__ __forceinline__ void dft_small<2>(float2* v, int, const float2* __restrict__, int) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void dft_small<4>(float2* v, int dir, const float2* __restrict__, int) {
  float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  float2 s13 = cadd(v[1], v[3]), d13 = cmul_mi(csub(v[1], v[3]), dir);
  v[0] = cadd(s02, s13);
  v[2] = csub(s02, s13);
  v[1] = cadd(d02, d13);
  v[3] = csub(d02, d13);
}

template <>
__device__ __forceinline__ void dft_small<8>(float2* v, int dir, const float2* __restrict__, int) {
  // radix-2 split into even/odd 4-point DFTs; W8 = exp(-i pi/4 * dir)
  const float h = 0.70710678118654752440f;
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft_small<4>(e, dir, nullptr, 0);
  dft_small<4>(o, dir, nullptr, 0);
  // o[r] *= W8^r
  float2 o1 = o[1];
  o[1] = make_float2(h * (o1.x + dir * o1.y), h * (o1.y - dir * o1.x));
  o[2] = cmul_mi(o[2], dir);
  float2 o3 = o[3];
  o[3] = make_float2(h * (-o3.x + dir * o3.y), h * (-o3.y - dir * o3.x));
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    v[r] = cadd(e[r], o[r]);
    v[r + 4] = csub(e[r], o[r]);
  }
}

// One Stockham stage with a compile-time radix.
template <int R>
__device__ __forceinline__ void stage_fixed(const float2* in, float2* out, int N, int Ns,
                                            const float2* __restrict__ tw, int dir, int nb,
                                            int sb, int sn, bool bfast, int tid, int nthr) {
  const int M = N / R;
  const int ts = N / (Ns * R);
  const int tot = M * nb;
  for (int w = tid; w < tot; w += nthr) {
    int b, j;
    if (bfast) { b = w % nb; j = w / nb; } else { j = w % M; b = w / M; }
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[b * sb + (j + r * M) * sn];
    const int k = j % Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twid(tw, k * r * ts, dir));
    }
    dft_small<R>(v, dir, tw, N);
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[b * sb + (base + r * Ns) * sn] = v[r];
  }
}

// Generic radix (odd primes of uneven scan sizes): direct O(R^2) DFT with
// W_R^{rs} = tw[(r s mod R) N/R].
__device__ __forceinline__ void stage_generic(const float2* in, float2* out, int N, int Ns, int R,
                                              const float2* __restrict__ tw, int dir, int nb, int sb,
                                              int sn, bool bfast, int tid, int nthr) {
  const int M = N / R;
  const int ts = N / (Ns * R);
  const int tot = M * nb;
  const int NR = N / R;
  for (int w = tid; w < tot; w += nthr) {
    int b, j;
    if (bfast) { b = w % nb; j = w / nb; } else { j = w % M; b = w / M; }
    const int k = j % Ns;
    const int base = (j / Ns) * Ns * R + k;
    for (int s = 0; s < R; ++s) {
      float2 acc = make_float2(0.f, 0.f);
      int e = 0;  // (r*s) mod R
      for (int r = 0; r < R; ++r) {
        float2 x = in[b * sb + (j + r * M) * sn];
        if (Ns > 1 && r > 0) x = cmul(x, twid(tw, k * r * ts, dir));
        acc = cadd(acc, cmul(x, twid(tw, e * NR, dir)));
        e += s;
        if (e >= R) e -= R;
      }
      out[b * sb + (base + s * Ns) * sn] = acc;
    }
  }
}

// Full transform on shared buffers A (input) and B (scratch); returns the
// buffer holding the result.  Must be called by all threads of the CTA.
__device__ __forceinline__ float2* fft_smem(float2* A, float2* B, const FftDesc& d, int dir, int nb,
                                            int sb, int sn, bool bfast) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  int Ns = 1;
  float2* in = A;
  float2* out = B;
  for (int s = 0; s < d.nst; ++s) {
    const int R = d.radix[s];
    switch (R) {
      case 2: stage_fixed<2>(in, out, d.N, Ns, d.tw, dir, nb, sb, sn, bfast, tid, nthr); break;
      case 4: stage_fixed<4>(in, out, d.N, Ns, d.tw, dir, nb, sb, sn, bfast, tid, nthr); break;
      case 8: stage_fixed<8>(in, out, d.N, Ns, d.tw, dir, nb, sb, sn, bfast, tid, nthr); break;
      default: stage_generic(in, out, d.N, Ns, R, d.tw, dir, nb, sb, sn, bfast, tid, nthr); break;
    }
    __syncthreads();
    float2* t = in;
    in = out;
    out = t;
    Ns *= R;
  }
  return in;
}
