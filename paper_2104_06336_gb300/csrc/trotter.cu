// Single-sideband integration (Sec. IV, set K and Eq. 3) with the probe
// aberration phase, fused in one kernel, and its adjoint with respect to the
// aberrations.
//
// Readings (the paper prints every vector of the set and of Eq. 3 as q):
//   K(K) = {k : |k| < k0, |k - K'| < k0, |k + K'| > k0}
//   S(K) = sum_{k in K(K)} G(k, K) exp(-i (chi(k) - chi(k - K')))   [/|K(K)|]
//   phi  = (N_R / Gbar0) Im(IFFT2(S)),   Gbar0 = mean_{k in BF} G(k, 0).
// Mask membership is decided in float32 with round-to-nearest products and
// sums (no fused multiply-add), K'x = c Kx0 - s Ky0, K'y = s Kx0 + c Ky0,
// Kx0 = m_x kpm_x, so an independent float32 evaluation gives the same set.
//
// G is stored for K_x >= 0 only: G[mx][my][p], G(k, -K) = conj G(k, K).  One
// warp handles one stored bin b and produces both S(b) (pixels of K(K'(b)),
// reading G(b)) and S(-b) (pixels of K(K'(-b)), reading conj G(b)), hence
//   H(b) = scale (S(b) - conj S(-b)) / (2 i),
// the transform of the real image phi: phi = IFFT2(H) with H Hermitian, so
// the inverse is a real (C2R) transform and V = sum_b |H(b)|^2 / N_R^2
// (Parseval).  The aberration-weighted spectrum is never written to memory.
//
// Per warp and bin: lanes own detector rows and compute, exactly, the integer
// kx intervals of each disk on their row, then write the member pixels of
// K(K'(b)) and K(K'(-b)) to two shared lists; lanes then stream the lists
// (consecutive pixels -> coalesced loads of G) and accumulate.
#include "common.cuh"

namespace {

constexpr float kTwoPi = 6.28318530717958647692f;

struct CandCoef {
  float a1, a2, a3, a4;  // chi/(2 pi) = a1 r2 + a2 (qx^2-qy^2) + a3 qx qy + a4 r2^2
  float c, s;            // float32 cos/sin of the rotation
  float u1, u3, u4;      // 2 pi dalpha^2/(2 lambda), 2 pi dalpha^2/lambda, 2 pi dalpha^4/(4 lambda)
  float pad[3];
};

struct TrotParams {
  int Ny, Nx, nkx, P_pad, n_rows, list_cap;
  float kpm_x, kpm_y, k0sq;
  int norm;
  int n_cand;
  float NR;
};

__device__ __forceinline__ float chi_turns(const CandCoef& c, float qx, float qy) {
  const float r2 = fmaf(qx, qx, qy * qy);
  const float ast = fmaf(c.a2, (qx - qy) * (qx + qy), c.a3 * (qx * qy));
  return fmaf(fmaf(c.a4, r2, c.a1), r2, ast);
}

// Candidate coefficients and per-pixel exp(-i chi(k_p)).
__global__ void k_prep(const double* __restrict__ aberr, int n_cand, const short2* __restrict__ pix,
                       int P_pad, int P, double dalpha, double lambda, CandCoef* coef, float2* ek,
                       uint32_t* st) {
  __shared__ CandCoef sc;
  const int c = blockIdx.x;
  if (threadIdx.x == 0) {
    const double* a = aberr + 5 * c;
    const double d2 = dalpha * dalpha;
    CandCoef k;
    k.a1 = (float)(a[0] * d2 / (2.0 * lambda));
    k.a2 = (float)(a[1] * d2 / (2.0 * lambda));
    k.a3 = (float)(a[2] * d2 / lambda);
    k.a4 = (float)(a[3] * d2 * d2 / (4.0 * lambda));
    k.c = (float)cos(aberr[4]);  // the mask rotation is that of candidate 0
    k.s = (float)sin(aberr[4]);
    const double tp = 6.283185307179586476925;
    k.u1 = (float)(tp * d2 / (2.0 * lambda));
    k.u3 = (float)(tp * d2 / lambda);
    k.u4 = (float)(tp * d2 * d2 / (4.0 * lambda));
    k.pad[0] = k.pad[1] = k.pad[2] = 0.f;
    if (a[4] != aberr[4]) st_or(st, EER4D_ST_ROTATION);
    sc = k;
    coef[c] = k;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < P_pad; p += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (p < P) {
      const short2 k = pix[p];
      const float t = chi_turns(sc, (float)k.x, (float)k.y);
      float sn, cs;
      sincospif(2.f * t, &sn, &cs);
      v = make_float2(cs, -sn);
    }
    ek[(size_t)c * P_pad + p] = v;
  }
}

// Gbar0 = mean over bright-field pixels of G(k, 0); scale = N_R / Gbar0.
__global__ void k_gbar(const float2* __restrict__ G, const int4* __restrict__ rows, int n_rows,
                       double NR, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  long long n = 0;
  for (int r = 0; r < n_rows; ++r) {
    const int4 R = rows[r];
    const int len = R.z - R.y + 1;
    for (int i = threadIdx.x; i < len; i += blockDim.x) s += (double)G[R.w + i].x;
    n += len;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double g0 = n ? red[0] / (double)n : 0.0;
    out[0] = g0;
    out[1] = g0 != 0.0 ? NR / g0 : 0.0;
  }
}

// integers x in [L, R] with d(x) = (x - c)^2 + dy2 (float32, rn) < thr
// (strict) or <= thr; the set is an interval, all of whose points lie in
// [ceil(c - r) - 1, floor(c + r) + 1], r = sqrt(max(thr - dy2, 0)).
__device__ __forceinline__ bool disk_pred(int x, float c, float dy2, float thr, bool strict) {
  const float dx = __fsub_rn((float)x, c);
  const float d = __fadd_rn(__fmul_rn(dx, dx), dy2);
  return strict ? (d < thr) : (d <= thr);
}
__device__ __forceinline__ void disk_interval(float c, float dy2, float thr, bool strict, int L,
                                              int R, int& a, int& b) {
  const float r2 = thr - dy2;
  const float r = r2 > 0.f ? sqrtf(r2) : 0.f;
  int a0 = max(L, (int)ceilf(c - r) - 1);
  int b0 = min(R, (int)floorf(c + r) + 1);
  while (a0 <= b0 && !disk_pred(a0, c, dy2, thr, strict)) ++a0;
  while (b0 >= a0 && !disk_pred(b0, c, dy2, thr, strict)) --b0;
  a = a0;
  b = b0;
}

// Member pixels of K(K') on row R (ky, lo, hi, p_lo): up to two segments.
__device__ __forceinline__ int row_segments(const int4 R, float Kx, float Ky, float k0sq, int& s0a,
                                            int& s0b, int& s1a, int& s1b) {
  const float dyi = __fsub_rn((float)R.x, Ky);
  const float dye = __fsub_rn((float)R.x, -Ky);
  int a2, b2, a3, b3;
  disk_interval(Kx, __fmul_rn(dyi, dyi), k0sq, true, R.y, R.z, a2, b2);
  s0a = 1; s0b = 0; s1a = 1; s1b = 0;
  if (a2 > b2) return 0;
  disk_interval(-Kx, __fmul_rn(dye, dye), k0sq, false, R.y, R.z, a3, b3);
  if (a3 > b3 || b3 < a2 || a3 > b2) {
    s0a = a2; s0b = b2;
  } else {
    s0a = a2; s0b = min(b2, a3 - 1);
    s1a = max(a2, b3 + 1); s1b = b2;
  }
  return max(0, s0b - s0a + 1) + max(0, s1b - s1a + 1);
}

__device__ __forceinline__ void kprime(const CandCoef& c0, float kpm_x, float kpm_y, int m_x,
                                       int m_y, float& Kx, float& Ky) {
  const float kx0 = __fmul_rn((float)m_x, kpm_x);
  const float ky0 = __fmul_rn((float)m_y, kpm_y);
  Kx = __fsub_rn(__fmul_rn(c0.c, kx0), __fmul_rn(c0.s, ky0));
  Ky = __fadd_rn(__fmul_rn(c0.s, kx0), __fmul_rn(c0.c, ky0));
}

// Builds list[0..n) of member pixels of K(K') for the warp (all lanes call).
__device__ __forceinline__ int build_list(const int4* __restrict__ srows, int n_rows, float Kx,
                                          float Ky, float k0sq, uint16_t* list) {
  const int lane = threadIdx.x & 31;
  int base = 0;
  for (int r0 = 0; r0 < n_rows; r0 += 32) {
    const int r = r0 + lane;
    int s0a = 1, s0b = 0, s1a = 1, s1b = 0, cnt = 0;
    int4 R = make_int4(0, 0, -1, 0);
    if (r < n_rows) {
      R = srows[r];
      cnt = row_segments(R, Kx, Ky, k0sq, s0a, s0b, s1a, s1b);
    }
    int total;
    int pos = base + warp_excl_scan(cnt, total);
    for (int x = s0a; x <= s0b; ++x) list[pos++] = (uint16_t)(R.w + (x - R.y));
    for (int x = s1a; x <= s1b; ++x) list[pos++] = (uint16_t)(R.w + (x - R.y));
    base += total;
  }
  __syncwarp();
  return base;
}

template <bool GRAD>
struct Acc {
  float2 S;
  float2 D[GRAD ? 5 : 1];
};

// Streams one list: term = g * exp(-i chi(k)) exp(+i chi(q)), q = k - K'.
template <bool GRAD, bool CONJ>
__device__ __forceinline__ void accumulate(const uint16_t* list, int n, const float2* __restrict__ Gb,
                                           const short2* __restrict__ spix,
                                           const float2* __restrict__ ekc, const CandCoef& cf,
                                           float Kx, float Ky, Acc<GRAD>& acc) {
  const int lane = threadIdx.x & 31;
  for (int j = lane; j < n; j += 32) {
    const int p = list[j];
    float2 g = __ldg(Gb + p);
    if (CONJ) g.y = -g.y;
    const short2 kk = spix[p];
    const float kx = (float)kk.x, ky = (float)kk.y;
    const float qx = kx - Kx, qy = ky - Ky;
    const float t = chi_turns(cf, qx, qy);
    float sn, cs;
    sincospif(2.f * t, &sn, &cs);
    const float2 e = __ldg(ekc + p);
    const float2 ph = make_float2(e.x * cs - e.y * sn, e.x * sn + e.y * cs);
    const float2 term = cmul(g, ph);
    acc.S = cadd(acc.S, term);
    if constexpr (GRAD) {
      const float r2k = fmaf(kx, kx, ky * ky), r2q = fmaf(qx, qx, qy * qy);
      const float d1 = cf.u1 * (r2k - r2q);
      const float d2 = cf.u1 * ((kx - ky) * (kx + ky) - (qx - qy) * (qx + qy));
      const float d3 = cf.u3 * (kx * ky - qx * qy);
      const float d4 = cf.u4 * (r2k * r2k - r2q * r2q);
      const float s4 = 4.f * cf.a4 * r2q;
      const float gx = fmaf(2.f * (cf.a1 + cf.a2) + s4, qx, cf.a3 * qy);
      const float gy = fmaf(2.f * (cf.a1 - cf.a2) + s4, qy, cf.a3 * qx);
      const float d5 = kTwoPi * (gy * Kx - gx * Ky);
      const float2 mi = make_float2(term.y, -term.x);  // -i * term
      acc.D[0] = make_float2(fmaf(d1, mi.x, acc.D[0].x), fmaf(d1, mi.y, acc.D[0].y));
      acc.D[1] = make_float2(fmaf(d2, mi.x, acc.D[1].x), fmaf(d2, mi.y, acc.D[1].y));
      acc.D[2] = make_float2(fmaf(d3, mi.x, acc.D[2].x), fmaf(d3, mi.y, acc.D[2].y));
      acc.D[3] = make_float2(fmaf(d4, mi.x, acc.D[3].x), fmaf(d4, mi.y, acc.D[3].y));
      acc.D[4] = make_float2(fmaf(d5, mi.x, acc.D[4].x), fmaf(d5, mi.y, acc.D[4].y));
    }
  }
}

__device__ __forceinline__ float2 warp_csum(float2 v) { return make_float2(warp_sum(v.x), warp_sum(v.y)); }

// H = scale (A/na - conj(B/nb)) / (2i), with A/n = 0 when n = 0 under area norm.
__device__ __forceinline__ float2 combine(float2 A, float2 B, int na, int nb, int norm, float scale) {
  if (norm) {
    A = na ? cscale(A, 1.f / (float)na) : make_float2(0.f, 0.f);
    B = nb ? cscale(B, 1.f / (float)nb) : make_float2(0.f, 0.f);
  }
  const float2 X = make_float2(A.x - B.x, A.y + B.y);  // A - conj(B)
  return make_float2(0.5f * scale * X.y, -0.5f * scale * X.x);
}

template <int MODE>
__global__ void __launch_bounds__(EER4D_WARPS_TROTTER * 32)
    k_trotter(TrotParams P, const float2* __restrict__ G, const short2* __restrict__ pix,
              const int4* __restrict__ rows, const CandCoef* __restrict__ coef,
              const float2* __restrict__ ek, const double* __restrict__ gscale,
              const float2* __restrict__ W, float2* H, double* partial, int32_t* count) {
  extern __shared__ unsigned char smem_raw[];
  short2* spix = reinterpret_cast<short2*>(smem_raw);
  int4* srows = reinterpret_cast<int4*>(spix + P.P_pad);
  uint16_t* lists = reinterpret_cast<uint16_t*>(srows + P.n_rows);
  constexpr bool GRAD = (MODE == TROT_GRAD || MODE == TROT_VARGRAD);
  constexpr int NV = GRAD ? 5 : 1;
  __shared__ double sred[EER4D_WARPS_TROTTER][5];

  for (int i = threadIdx.x; i < P.P_pad; i += blockDim.x) spix[i] = pix[i];
  for (int i = threadIdx.x; i < P.n_rows; i += blockDim.x) srows[i] = rows[i];
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint16_t* listP = lists + (size_t)warp * 2 * P.list_cap;
  uint16_t* listM = listP + P.list_cap;
  const CandCoef c0 = coef[0];
  const float scale = (float)gscale[1];
  const int ntask = P.nkx * P.Ny;
  const int gw = blockIdx.x * EER4D_WARPS_TROTTER + warp;
  const int nwarps = gridDim.x * EER4D_WARPS_TROTTER;
  double gacc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) gacc[j] = 0.0;

  for (int t = gw; t < ntask; t += nwarps) {
    const int mx = t / P.Ny, my = t - mx * P.Ny;
    const int mmx = (P.Nx - mx) % P.Nx, mmy = (P.Ny - my) % P.Ny;
    float Kpx, Kpy, Kmx, Kmy;
    kprime(c0, P.kpm_x, P.kpm_y, freq_index(mx, P.Nx), freq_index(my, P.Ny), Kpx, Kpy);
    kprime(c0, P.kpm_x, P.kpm_y, freq_index(mmx, P.Nx), freq_index(mmy, P.Ny), Kmx, Kmy);
    const int nP = build_list(srows, P.n_rows, Kpx, Kpy, P.k0sq, listP);
    const int nM = build_list(srows, P.n_rows, Kmx, Kmy, P.k0sq, listM);
    if (MODE == TROT_COUNT) {
      if (lane == 0) {
        count[my * P.Nx + mx] = nP;
        count[mmy * P.Nx + mmx] = nM;
      }
      __syncwarp();
      continue;
    }
    const float2* Gb = G + (size_t)t * P.P_pad;
    const float wgt = (mx == 0 || 2 * mx == P.Nx) ? 1.f : 2.f;
    const int nc = (MODE == TROT_FWD) ? P.n_cand : 1;
    for (int c = 0; c < nc; ++c) {
      const CandCoef cf = (c == 0) ? c0 : coef[c];
      const float2* ekc = ek + (size_t)c * P.P_pad;
      Acc<GRAD> ap, am;
      ap.S = am.S = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < (GRAD ? 5 : 1); ++j) ap.D[j] = am.D[j] = make_float2(0.f, 0.f);
      accumulate<GRAD, false>(listP, nP, Gb, spix, ekc, cf, Kpx, Kpy, ap);
      accumulate<GRAD, true>(listM, nM, Gb, spix, ekc, cf, Kmx, Kmy, am);
      ap.S = warp_csum(ap.S);
      am.S = warp_csum(am.S);
      const float2 Hb = combine(ap.S, am.S, nP, nM, P.norm, scale);
      if (MODE != TROT_GRAD && lane == 0) H[((size_t)c * P.Ny + my) * P.nkx + mx] = Hb;
      if constexpr (GRAD) {
        float2 wb;
        double f;
        if (MODE == TROT_VARGRAD) {  // dV/dtheta: w = 2 H / N_R, factor 1/N_R
          wb = Hb;
          f = 2.0 / ((double)P.NR * (double)P.NR);
        } else {
          wb = __ldg(W + (size_t)my * P.nkx + mx);
          f = 1.0 / (double)P.NR;
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          const float2 dp = warp_csum(ap.D[j]);
          const float2 dm = warp_csum(am.D[j]);
          const float2 dH = combine(dp, dm, nP, nM, P.norm, scale);
          // Re(dH * conj(w))
          const double re = (double)dH.x * (double)wb.x + (double)dH.y * (double)wb.y;
          gacc[j] += (double)wgt * f * re;
        }
      }
    }
  }
  if constexpr (GRAD) {
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < NV; ++j) sred[warp][j] = gacc[j];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
      double s = 0.0;
      for (int w = 0; w < EER4D_WARPS_TROTTER; ++w) s += sred[w][threadIdx.x];
      partial[(size_t)blockIdx.x * NV + threadIdx.x] = s;
    }
  }
}

// Fixed-order sum of per-block partials (deterministic).
__global__ void k_reduce_partials(const double* partial, int nblk, int nv, double* out) {
  __shared__ double red[256];
  for (int j = 0; j < nv; ++j) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(size_t)b * nv + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = red[0];
    __syncthreads();
  }
}

// V_c = sum_b w(b) |H_c(b)|^2 / N_R^2 over the stored half: per-block partial
// sums (grid kVarBlocks x n_cand), then a fixed-order final sum per candidate.
constexpr int kVarBlocks = 128;

__global__ void k_variance_partial(const float2* __restrict__ H, int Ny, int nkx, int Nx,
                                   double* part) {
  __shared__ double red[256];
  const int c = blockIdx.y;
  const float2* h = H + (size_t)c * Ny * nkx;
  double s = 0.0;
  const int n = Ny * nkx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int mx = i % nkx;
    const double w = (mx == 0 || 2 * mx == Nx) ? 1.0 : 2.0;
    const float2 v = h[i];
    s += w * ((double)v.x * v.x + (double)v.y * v.y);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)c * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_variance_final(const double* __restrict__ part, int nblk, double NR, double* var) {
  __shared__ double red[128];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(size_t)c * nblk + b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) var[c] = red[0] / (NR * NR);
}

__global__ void k_ascent(double* theta, const double* step, const double* grad) {
  const int j = threadIdx.x;
  if (j < 5) theta[j] += step[j] * grad[j];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int trot_blocks(const eer4d_plan* p) {
  const int ntask = p->nkx * (int)p->g.scan_ny;
  int b = (ntask + EER4D_WARPS_TROTTER - 1) / EER4D_WARPS_TROTTER;
  return b < 152 * 8 ? b : 152 * 8;
}

struct Layout {
  size_t coef, ek, gscale, H, partial, vpart, total;
};
Layout layout(const eer4d_plan* p, int n_cand, int mode) {
  Layout L;
  size_t o = 0;
  L.coef = o; o = align256(o + sizeof(CandCoef) * n_cand);
  L.ek = o; o = align256(o + sizeof(float2) * (size_t)n_cand * p->P_pad);
  L.gscale = o; o = align256(o + 2 * sizeof(double));
  const int nh = (mode == TROT_GRAD || mode == TROT_COUNT) ? 0 : n_cand;
  L.H = o; o = align256(o + sizeof(float2) * (size_t)nh * p->g.scan_ny * p->nkx);
  L.partial = o; o = align256(o + sizeof(double) * 5 * trot_blocks(p));
  L.vpart = o; o = align256(o + sizeof(double) * kVarBlocks * (size_t)nh);
  L.total = o;
  return L;
}

}  // namespace

cudaError_t launch_ascent(double* theta, const double* step, const double* grad, cudaStream_t s) {
  k_ascent<<<1, 32, 0, s>>>(theta, step, grad);
  count_launches(1);
  return cudaGetLastError();
}

size_t trotter_scratch_bytes(const eer4d_plan* p, int n_cand, int mode) {
  return layout(p, n_cand, mode).total;
}

cudaError_t launch_trotter(const eer4d_plan* p, const float2* G, const double* aberr, int n_cand,
                           int mode, void* scratch, const float2* W, float* phase_out,
                           double* var_out, double* grad_out, int32_t* count_out, uint32_t* st,
                           cudaStream_t s) {
  const Layout L = layout(p, n_cand, mode);
  unsigned char* sb = static_cast<unsigned char*>(scratch);
  CandCoef* coef = reinterpret_cast<CandCoef*>(sb + L.coef);
  float2* ek = reinterpret_cast<float2*>(sb + L.ek);
  double* gsc = reinterpret_cast<double*>(sb + L.gscale);
  float2* H = reinterpret_cast<float2*>(sb + L.H);
  double* partial = reinterpret_cast<double*>(sb + L.partial);
  double* vpart = reinterpret_cast<double*>(sb + L.vpart);
  cudaError_t e;
  stage_begin(p, EER4D_STAGE_TROTTER, s);
  k_prep<<<n_cand, 256, 0, s>>>(aberr, n_cand, p->d_pix, p->P_pad, p->P, p->g.dalpha_rad,
                                p->g.lambda_A, coef, ek, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (mode != TROT_COUNT) {
    k_gbar<<<1, 256, 0, s>>>(G, p->d_rows, p->n_rows, (double)p->F, gsc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  TrotParams tp;
  tp.Ny = p->g.scan_ny; tp.Nx = p->g.scan_nx; tp.nkx = p->nkx; tp.P_pad = p->P_pad;
  tp.n_rows = p->n_rows; tp.list_cap = p->list_max;
  tp.kpm_x = (float)p->g.kpm_x; tp.kpm_y = (float)p->g.kpm_y;
  tp.k0sq = (float)(p->g.k0_px * p->g.k0_px);
  tp.norm = p->norm; tp.n_cand = n_cand; tp.NR = (float)p->F;
  const size_t sm = sizeof(short2) * p->P_pad + sizeof(int4) * p->n_rows +
                    sizeof(uint16_t) * 2 * (size_t)p->list_max * EER4D_WARPS_TROTTER;
  const int nblk = trot_blocks(p);
  const dim3 blk(EER4D_WARPS_TROTTER * 32);
#define EER4D_LAUNCH_TROT(M)                                                                       \
  do {                                                                                            \
    if ((e = ensure_smem((const void*)k_trotter<M>, sm)) != cudaSuccess) return e;               \
    k_trotter<M><<<nblk, blk, sm, s>>>(tp, G, p->d_pix, p->d_rows, coef, ek, gsc, W, H, partial, \
                                       count_out);                                                \
  } while (0)
  switch (mode) {
    case TROT_FWD: EER4D_LAUNCH_TROT(TROT_FWD); break;
    case TROT_GRAD: EER4D_LAUNCH_TROT(TROT_GRAD); break;
    case TROT_VARGRAD: EER4D_LAUNCH_TROT(TROT_VARGRAD); break;
    default: EER4D_LAUNCH_TROT(TROT_COUNT); break;
  }
#undef EER4D_LAUNCH_TROT
  count_launches(mode == TROT_COUNT ? 2 : 3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (mode == TROT_GRAD || mode == TROT_VARGRAD) {
    k_reduce_partials<<<1, 256, 0, s>>>(partial, nblk, 5, grad_out);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  stage_end(p, EER4D_STAGE_TROTTER, s);
  if (mode == TROT_COUNT || mode == TROT_GRAD) return cudaSuccess;
  const int nc = mode == TROT_FWD ? n_cand : 1;
  stage_begin(p, EER4D_STAGE_IMAGE, s);
  if (var_out) {
    k_variance_partial<<<dim3(kVarBlocks, nc), 256, 0, s>>>(H, p->g.scan_ny, p->nkx, p->g.scan_nx,
                                                             vpart);
    k_variance_final<<<nc, 128, 0, s>>>(vpart, kVarBlocks, (double)p->F, var_out);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (phase_out && (e = launch_c2r_image(p, H, phase_out, nc, s)) != cudaSuccess) return e;
  stage_end(p, EER4D_STAGE_IMAGE, s);
  return cudaSuccess;
}
