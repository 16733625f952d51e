// Single-sideband integration (Sec. IV, set K and Eq. 3) with the probe
// aberration phase, fused in one kernel, and its adjoint with respect to the
// aberrations.
//
// Readings (the paper prints every vector of the set and of Eq. 3 as q):
//   K(K) = {k : |k| < k0, |k - K'| < k0, |k + K'| > k0}
//   S(K) = sum_{k in K(K)} G(k, K) exp(-i (chi(k) - chi(k - K')))   [/|K(K)|]
//   phi  = (N_R / Gbar0) Im(IFFT2(S)),   Gbar0 = mean_{k in BF} G(k, 0).
// Mask membership is decided in float32 with round-to-nearest products and
// sums (no fused multiply-add): K'x = c Kx0 - s Ky0, K'y = s Kx0 + c Ky0,
// Kx0 = m_x kpm_x, d(k, K') = (kx - K'x)^2 + (ky - K'y)^2, so an independent
// float32 evaluation in the same order gives the same set.
//
// G is stored for K_x >= 0 only, with K_y innermost: G[mx][p][my],
// G(k, -K) = conj G(k, K).  A warp owns 32 consecutive stored bins
// b = (mx, my0 .. my0+31), one per lane, and walks the bright-field pixels:
// for each pixel every lane decides membership of its own bin's two sets,
// K(K'(b)) (reads G(k, b)) and K(K'(-b)) (reads conj G(k, b)); a pixel's
// G values of the 32 bins are one contiguous 256-byte row, and nearby bins
// have nearly the same sets, so loads are coalesced and whole sectors are
// used.  Each lane ends with
//   H(b) = scale (S(b) - conj S(-b)) / (2 i),
// the transform of the real image phi: phi = IFFT2(H) with H Hermitian, so
// the inverse is a real (C2R) transform and V = sum_b |H(b)|^2 / N_R^2
// (Parseval).  The aberration-weighted spectrum is never written to memory.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace {

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr int kWarps = EER4D_WARPS_TROTTER;
constexpr int kBatch = 8;  // pixels per batch of the trotter pixel loop

struct CandCoef {
  float a1, a2, a3, a4;  // chi/(2 pi) = a1 r2 + a2 (qx^2-qy^2) + a3 qx qy + a4 r2^2
  float c, s;            // float32 cos/sin of the rotation
  float u1, u3, u4;      // 2 pi dalpha^2/(2 lambda), 2 pi dalpha^2/lambda, 2 pi dalpha^4/(4 lambda)
  float pad[3];
};

struct TrotParams {
  int Ny, Nx, nkx, P_pad, P_bf;
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
// own_rot: every row uses its own rotation (independent datasets); otherwise
// the mask rotation of all candidates is that of row 0 and a different
// rotation in another row is flagged.
__global__ void k_prep(const double* __restrict__ aberr, int n_cand, const short2* __restrict__ pix,
                       int P_pad, int P, double dalpha, double lambda, CandCoef* coef, float2* ek,
                       uint32_t* st, int own_rot = 0, unsigned* qctr = nullptr) {
  __shared__ CandCoef sc;
  const int c = blockIdx.x;
  if (qctr && threadIdx.x == 0) qctr[c] = 0u;  // the work queue of candidate pass c
  if (threadIdx.x == 0) {
    const double* a = aberr + 5 * c;
    const double d2 = dalpha * dalpha;
    CandCoef k;
    k.a1 = (float)(a[0] * d2 / (2.0 * lambda));
    k.a2 = (float)(a[1] * d2 / (2.0 * lambda));
    k.a3 = (float)(a[2] * d2 / lambda);
    k.a4 = (float)(a[3] * d2 * d2 / (4.0 * lambda));
    const double rot = own_rot ? a[4] : aberr[4];
    k.c = (float)cos(rot);
    k.s = (float)sin(rot);
    const double tp = 6.283185307179586476925;
    k.u1 = (float)(tp * d2 / (2.0 * lambda));
    k.u3 = (float)(tp * d2 / lambda);
    k.u4 = (float)(tp * d2 * d2 / (4.0 * lambda));
    k.pad[0] = k.pad[1] = k.pad[2] = 0.f;
    if (!own_rot && a[4] != aberr[4]) st_or(st, EER4D_ST_ROTATION);
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
// G(k_p, 0) sits at G[0][p][0] = G[p * Ny].
__global__ void k_gbar(const float2* __restrict__ G, const int32_t* __restrict__ bfp, int P_bf,
                       int Ny, double NR, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int q = threadIdx.x; q < P_bf; q += blockDim.x) s += (double)G[(size_t)bfp[q] * Ny].x;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double g0 = P_bf ? red[0] / (double)P_bf : 0.0;
    out[0] = g0;
    out[1] = g0 != 0.0 ? NR / g0 : 0.0;
  }
}

__device__ __forceinline__ void kprime(const CandCoef& c0, float kpm_x, float kpm_y, int m_x,
                                       int m_y, float& Kx, float& Ky) {
  const float kx0 = __fmul_rn((float)m_x, kpm_x);
  const float ky0 = __fmul_rn((float)m_y, kpm_y);
  Kx = __fsub_rn(__fmul_rn(c0.c, kx0), __fmul_rn(c0.s, ky0));
  Ky = __fadd_rn(__fmul_rn(c0.s, kx0), __fmul_rn(c0.c, ky0));
}

// |k - K|^2 in float32, round-to-nearest, products then sum (the mask rule)
__device__ __forceinline__ float dist2(float kx, float ky, float Kx, float Ky) {
  const float dx = __fsub_rn(kx, Kx), dy = __fsub_rn(ky, Ky);
  return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// Membership of detector pixel kk in the bin's two sets (the exact float32
// rule): memP for K(K'(b)), memM for K(K'(-b)); off Nyquist K'(-b) = -K'(b)
// and the two distances serve both sets.
__device__ __forceinline__ void member_bits(float2 kk, float Kpx, float Kpy, float Kmx, float Kmy,
                                            bool nyq, bool active, float k0sq, bool& memP,
                                            bool& memM) {
  const float dm = dist2(kk.x, kk.y, Kpx, Kpy);
  const float dp = dist2(kk.x, kk.y, -Kpx, -Kpy);
  memP = active && dm < k0sq && dp > k0sq;
  if (!nyq) {
    memM = active && dp < k0sq && dm > k0sq;
  } else {
    const float em = dist2(kk.x, kk.y, Kmx, Kmy);
    const float ep = dist2(kk.x, kk.y, -Kmx, -Kmy);
    memM = active && em < k0sq && ep > k0sq;
  }
}

__device__ __forceinline__ float2 cmadd(float2 acc, float2 a, float w) {
  return make_float2(fmaf(w, a.x, acc.x), fmaf(w, a.y, acc.y));
}

// H = scale (A/na - conj(B/nb)) / (2i), with A/n = 0 when n = 0 under area norm.
__device__ __forceinline__ float2 combine(float2 A, float2 B, int na, int nb, int norm, float scale) {
  if (norm) {
    A = na ? cscale(A, 1.f / (float)na) : make_float2(0.f, 0.f);
    B = nb ? cscale(B, 1.f / (float)nb) : make_float2(0.f, 0.f);
  }
  const float2 X = make_float2(A.x - B.x, A.y + B.y);  // A - conj(B)
  return make_float2(0.5f * scale * X.y, -0.5f * scale * X.x);
}

// MODE: TROT_FWD (H for NC candidates per pass), TROT_GRAD (adjoint against
// W = FFT(upstream gradient)), TROT_VARGRAD (V and dV/dtheta), TROT_COUNT
// (|K(K)| per bin).
// Register budgets: one candidate at 3 CTAs per SM (80 registers); several
// candidates per pass (NC phase chains per term) and the gradient modes at 2,
// so that their per-candidate sums stay in registers instead of spilling.
template <int MODE, int NC, bool SPREAD = false>
__global__ void __launch_bounds__(kWarps * 32,
                                  (MODE == TROT_GRAD || MODE == TROT_VARGRAD || NC > 1) ? 2 : 3)
    k_trotter(TrotParams P, const float2* __restrict__ G, const int32_t* __restrict__ bfp,
              const short2* __restrict__ pix, const CandCoef* __restrict__ coef,
              const float2* __restrict__ ek, const double* __restrict__ gscale,
              const float2* __restrict__ W, float2* H, double* partial, int32_t* count,
              const uint32_t* __restrict__ tl_bits, const uint32_t* __restrict__ tl_qp,
              const int* __restrict__ tl_n, const int* __restrict__ tl_order, int tl_cap,
              unsigned* qctr, uint32_t* st) {
  constexpr bool GRAD = (MODE == TROT_GRAD || MODE == TROT_VARGRAD);
  extern __shared__ unsigned char smem_raw[];
  float2* skk = reinterpret_cast<float2*>(smem_raw);                  // [P_bf] (kx, ky)
  int* sp = reinterpret_cast<int*>(skk + P.P_bf);                      // [P_bf] kept-pixel index
  float2* sek = reinterpret_cast<float2*>(sp + ((P.P_bf + 1) & ~1));  // [NC][P_bf]

  for (int q = threadIdx.x; q < P.P_bf; q += blockDim.x) {
    const int p = bfp[q];
    const short2 k = pix[p];
    skk[q] = make_float2((float)k.x, (float)k.y);
    sp[q] = p;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const CandCoef c0 = coef[0];
  // the plan's membership lists hold the sets at scan rotation 0
  const bool lists = tl_n != nullptr && c0.c == 1.f && c0.s == 0.f;
  const float scale = MODE == TROT_COUNT ? 0.f : (float)gscale[1];
  const int nyw = (P.Ny + 31) >> 5;
  const int ntask = P.nkx * nyw;
  const int gw = blockIdx.x * kWarps + warp;
  const int nwarps = gridDim.x * kWarps;
  const int npass = (MODE == TROT_FWD) ? (P.n_cand + NC - 1) / NC : 1;

  // passes of NC candidates; SPREAD: blockIdx.y takes passes y, y + gridDim.y,
  // ... (a grid with more residency than one pass's warp tasks spreads the
  // passes over CTAs; without it the loop stays the plain one, which the
  // compiler schedules better)
  for (int pass = SPREAD ? (int)blockIdx.y : 0; pass < npass; pass += SPREAD ? (int)gridDim.y : 1) {
    const int cb = pass * NC;
    const int ncp = (MODE == TROT_FWD) ? min(NC, P.n_cand - cb) : 1;
    __syncthreads();
    if (MODE != TROT_COUNT) {
      for (int i = threadIdx.x; i < ncp * P.P_bf; i += blockDim.x) {
        const int c = i / P.P_bf, q = i - c * P.P_bf;
        sek[c * P.P_bf + q] = ek[(size_t)(cb + c) * P.P_pad + sp[q]];
      }
    }
    __syncthreads();
    CandCoef cf[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) cf[c] = coef[cb + (c < ncp ? c : 0)];

    // Warp tasks come from a work queue per candidate pass (with the lists,
    // longest first), so the warps of a pass finish together; without a
    // queue warp gw takes tasks gw, gw + nwarps, ...  A bin's sums never
    // leave its warp, and the gradient sums do not depend on the schedule
    // either: each task's share is stored at the task's index.
    const bool dyn = qctr != nullptr;
    auto take = [&]() -> int {
      unsigned v = 0u;
      if (lane == 0) v = atomicAdd(qctr + pass, 1u);
      return (int)__shfl_sync(0xffffffffu, v, 0);
    };
    const int* order = (dyn && lists) ? tl_order : nullptr;
    for (int u = dyn ? take() : gw; u < ntask; u = dyn ? take() : u + nwarps) {
      const int t = order ? __ldg(order + u) : u;
      if (!EER4D_IN_RANGE(t, ntask, st)) continue;  // warp-uniform (t is the warp's task)
      const int mx = t / nyw;
      const int my = (t - mx * nyw) * 32 + lane;
      const bool active = my < P.Ny;
      const int mys = active ? my : 0;
      const int mmx = (P.Nx - mx) % P.Nx, mmy = (P.Ny - mys) % P.Ny;
      float Kpx, Kpy, Kmx, Kmy;
      kprime(c0, P.kpm_x, P.kpm_y, freq_index(mx, P.Nx), freq_index(mys, P.Ny), Kpx, Kpy);
      kprime(c0, P.kpm_x, P.kpm_y, freq_index(mmx, P.Nx), freq_index(mmy, P.Ny), Kmx, Kmy);
      // off Nyquist K'(-b) = -K'(b) exactly and both sets use the same two distances
      const bool nyq = (2 * mx == P.Nx) || (2 * mys == P.Ny);
      const float2* Gl = G + (size_t)mx * P.P_pad * P.Ny + mys;
      float2 SP[NC], SM[NC];
      float2 DP[GRAD ? 5 : 1], DM[GRAD ? 5 : 1];
#pragma unroll
      for (int c = 0; c < NC; ++c) SP[c] = SM[c] = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < (GRAD ? 5 : 1); ++j) DP[j] = DM[j] = make_float2(0.f, 0.f);
      int nP = 0, nM = 0;
      // the warp's bins include a Nyquist bin (uniform across the warp, no intrinsic)
      const int my0 = (t - mx * nyw) * 32;
      const bool nyq_warp = (2 * mx == P.Nx) || (P.Ny / 2 >= my0 && P.Ny / 2 < my0 + 32);
      // one pair (k_q, b) of one set: term = g exp(-i chi(k)) exp(+i chi(k - K)),
      // added to S(b) with weight wp and to S(-b) with weight 1 - wp
      auto contrib = [&](float2 g, float Kx, float Ky, float2 kk, int q, float wp,
                         float2 (&SPa)[NC], float2 (&SMa)[NC], float2 (&DPa)[GRAD ? 5 : 1],
                         float2 (&DMa)[GRAD ? 5 : 1]) {
        const float qx = kk.x - Kx, qy = kk.y - Ky;
        const float wm = 1.f - wp;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if (c >= ncp) break;
          const float tq = chi_turns(cf[c], qx, qy);
          const float fr = tq - rintf(tq);  // exact: phase in turns reduced to [-1/2, 1/2]
          float sn, cs;
          __sincosf(kTwoPi * fr, &sn, &cs);
          const float2 e = sek[c * P.P_bf + q];
          const float2 ph = make_float2(e.x * cs - e.y * sn, e.x * sn + e.y * cs);
          const float2 term = cmul(g, ph);
          SPa[c] = cmadd(SPa[c], term, wp);
          SMa[c] = cmadd(SMa[c], term, wm);
          if constexpr (GRAD) {
            const CandCoef& f = cf[0];
            const float kx = kk.x, ky = kk.y;
            const float r2k = fmaf(kx, kx, ky * ky), r2q = fmaf(qx, qx, qy * qy);
            float d[5];
            d[0] = f.u1 * (r2k - r2q);
            d[1] = f.u1 * ((kx - ky) * (kx + ky) - (qx - qy) * (qx + qy));
            d[2] = f.u3 * (kx * ky - qx * qy);
            d[3] = f.u4 * (r2k * r2k - r2q * r2q);
            const float s4 = 4.f * f.a4 * r2q;
            const float gx = fmaf(2.f * (f.a1 + f.a2) + s4, qx, f.a3 * qy);
            const float gy = fmaf(2.f * (f.a1 - f.a2) + s4, qy, f.a3 * qx);
            d[4] = kTwoPi * (gy * Kx - gx * Ky);
            const float2 mi = make_float2(term.y, -term.x);  // -i * term
            if (P.norm == 0) {
              // Eq. 3 as printed needs only the difference A - conj(B): one
              // signed sum per parameter (wp = 1: the term, wp = 0: minus its
              // conjugate)
              const float sg = wp - wm;
#pragma unroll
              for (int j = 0; j < 5; ++j) {
                DPa[j].x = fmaf(sg * d[j], mi.x, DPa[j].x);
                DPa[j].y = fmaf(d[j], mi.y, DPa[j].y);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 5; ++j) {
                DPa[j] = cmadd(DPa[j], mi, d[j] * wp);
                DMa[j] = cmadd(DMa[j], mi, d[j] * wm);
              }
            }
          }
        }
      };

      // A batch of kBatch bright-field pixels with this lane's membership bits:
      // every member's G load is issued before any is used (kBatch loads in
      // flight).  Entry xv[i] is q << 16 | p (bright-field index, kept pixel)
      // from the lists (PACKED), or the index q itself.
      auto batch = [&](unsigned mP, unsigned mM, const uint32_t (&xv)[kBatch], auto packed) {
        constexpr bool PACKED = decltype(packed)::value;
        nP += __popc(mP);
        nM += __popc(mM);
        if (MODE == TROT_COUNT) return;
        const unsigned mAny = mP | mM;
        if (mAny == 0u) return;
        float2 gb[kBatch];
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
          float2 v = make_float2(0.f, 0.f);
          if ((mAny >> i) & 1u) {
            const int qi = PACKED ? (int)(xv[i] >> 16) : (int)xv[i];
            if (EER4D_IN_RANGE(qi, P.P_bf, st)) {
              const int prow = PACKED ? (int)(xv[i] & 0xffffu) : sp[qi];
              if (EER4D_IN_RANGE(prow, P.P_pad, st)) v = Gl[(size_t)prow * P.Ny];
            }
          }
          gb[i] = v;
        }
        if (PACKED && !nyq_warp) {
          // every list entry has a member among the warp's lanes, and a lane
          // that is not a member of entry i holds G = 0 there, so its term is
          // exactly 0: the entries run as independent straight-line chains
#pragma unroll
          for (int i = 0; i < kBatch; ++i) {
            const bool memM = (mM >> i) & 1u;
            int q = (int)(xv[i] >> 16);
#ifdef EER4D_CHECKS
            if (q >= P.P_bf) q = 0;  // its G is 0 (checked above): the term is 0
#endif
            const float2 g = gb[i];
            const float2 gg = memM ? make_float2(g.x, -g.y) : g;
            contrib(gg, memM ? Kmx : Kpx, memM ? Kmy : Kpy, skk[q], q, memM ? 0.f : 1.f, SP, SM, DP,
                    DM);
          }
          return;
        }
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
          const bool memP = (mP >> i) & 1u, memM = (mM >> i) & 1u;
          if (!(memP || memM)) continue;
          int q = PACKED ? (int)(xv[i] >> 16) : (int)xv[i];
#ifdef EER4D_CHECKS
          if (q >= P.P_bf) q = 0;  // its G is 0 (checked above): the term is 0
#endif
          const float2 kk = skk[q];
          const float2 g = gb[i];
          // Off Nyquist the two sets are disjoint, so one term per pixel: G into
          // S(b) or conj(G) into S(-b).  At a Nyquist bin K'(-b) equals K'(b) in
          // that component and a pixel may be in both sets: two terms.
          if (!nyq_warp) {
            const float2 gg = memM ? make_float2(g.x, -g.y) : g;
            contrib(gg, memM ? Kmx : Kpx, memM ? Kmy : Kpy, kk, q, memM ? 0.f : 1.f, SP, SM, DP, DM);
          } else {
            if (memP) contrib(g, Kpx, Kpy, kk, q, 1.f, SP, SM, DP, DM);
            if (memM) contrib(make_float2(g.x, -g.y), Kmx, Kmy, kk, q, 0.f, SP, SM, DP, DM);
          }
        }
      };
      if (lists) {
        // only the pixels with a member among the warp's bins, in ascending
        // q (the same sums in the same order), 32 entries at a time: each
        // lane reads its own two membership words (bit i = entry e0 + i) and
        // one packed (q, p) entry, which the shuffles hand to every lane
        int n = tl_n[t];
        if (!EER4D_IN_RANGE(n, tl_cap + 1, st)) n = 0;
        const uint32_t* bits = tl_bits + (size_t)t * (tl_cap / 32) * 64;
        const uint32_t* qps = tl_qp + (size_t)t * tl_cap;
        for (int e0 = 0; e0 < n; e0 += 32) {
          const uint32_t wP = __ldg(bits + 2 * e0 + lane);
          const uint32_t wM = __ldg(bits + 2 * e0 + 32 + lane);
          const uint32_t ql = __ldg(qps + e0 + lane);  // tl_cap is a multiple of 32
          const int m = n - e0 < 32 ? n - e0 : 32;
          for (int s0 = 0; s0 < m; s0 += kBatch) {
            uint32_t xv[kBatch];
#pragma unroll
            for (int i = 0; i < kBatch; ++i) xv[i] = __shfl_sync(0xffffffffu, ql, s0 + i);
            batch((wP >> s0) & 0xffu, (wM >> s0) & 0xffu, xv, std::true_type{});
          }
        }
      } else {
        for (int q0 = 0; q0 < P.P_bf; q0 += kBatch) {
          unsigned mP = 0u, mM = 0u;
          uint32_t xv[kBatch];
#pragma unroll
          for (int i = 0; i < kBatch; ++i) {
            const int q = q0 + i;
            xv[i] = q < P.P_bf ? q : 0;
            if (q >= P.P_bf) continue;
            bool memP, memM;
            member_bits(skk[q], Kpx, Kpy, Kmx, Kmy, nyq, active, P.k0sq, memP, memM);
            mP |= (unsigned)memP << i;
            mM |= (unsigned)memM << i;
          }
          batch(mP, mM, xv, std::false_type{});
        }
      }

      if constexpr (GRAD) {
        // this task's share of dV/dtheta, one bin per lane, stored at
        // (task, lane): the sum over tasks and lanes runs afterwards in a
        // fixed order, whatever warp took the task
        double tv[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (active) {
          const float wgt = (mx == 0 || 2 * mx == P.Nx) ? 1.f : 2.f;
          const float2 Hb = combine(SP[0], SM[0], nP, nM, P.norm, scale);
          if (MODE != TROT_GRAD) H[(size_t)my * P.nkx + mx] = Hb;
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
            const float2 dH = combine(DP[j], DM[j], nP, nM, P.norm, scale);
            tv[j] = (double)wgt * f * ((double)dH.x * (double)wb.x + (double)dH.y * (double)wb.y);
          }
        }
        double* dst = partial + ((size_t)t * 32 + lane) * 5;
#pragma unroll
        for (int j = 0; j < 5; ++j) dst[j] = tv[j];
      } else {
        if (!active) continue;
        if constexpr (MODE == TROT_COUNT) {
          count[my * P.Nx + mx] = nP;
          count[mmy * P.Nx + mmx] = nM;
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if (c >= ncp) break;
            const float2 Hb = combine(SP[c], SM[c], nP, nM, P.norm, scale);
            H[((size_t)(cb + c) * P.Ny + my) * P.nkx + mx] = Hb;
          }
        }
      }
    }
  }
}

// ---- several datasets of one detector geometry in one launch ---------------
// Every dataset s has its own scan (Ny, Nx), G, aberrations (row s of the
// candidates) and output spectrum H_s; the bright-field pixel table is shared.
// The warp tasks of all datasets are numbered one after another (task0 is the
// first of dataset s) and the persistent grid walks them all, so small scans
// fill the GPU together.  Same per-bin arithmetic, in the same pixel order, as
// the single-dataset kernel with one candidate.
constexpr int kMaxSets = EER4D_MAX_SETS;

struct SetDesc {
  const float2* G;
  float2* H;
  int Ny, Nx, nkx, norm;
  float kpm_x, kpm_y;
  int task0;
  float NR;
  // the dataset plan's membership lists (scan rotation 0), or tl_n = nullptr
  const uint32_t* tl_bits;
  const uint32_t* tl_qp;
  const int* tl_n;
  int tl_cap;
};

struct BatchParams {
  int n_sets, P_pad, P_bf, ntask;
  float k0sq;
  SetDesc s[kMaxSets];
};

__global__ void k_gbar_batched(const __grid_constant__ BatchParams B, const int32_t* __restrict__ bfp,
                               double* gscale) {
  __shared__ double red[256];
  const SetDesc& D = B.s[blockIdx.x];
  double sum = 0.0;
  for (int q = threadIdx.x; q < B.P_bf; q += blockDim.x) sum += (double)D.G[(size_t)bfp[q] * D.Ny].x;
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double g0 = B.P_bf ? red[0] / (double)B.P_bf : 0.0;
    gscale[2 * blockIdx.x] = g0;
    gscale[2 * blockIdx.x + 1] = g0 != 0.0 ? (double)D.NR / g0 : 0.0;
  }
}

__global__ void __launch_bounds__(kWarps * 32, 3)
    k_trotter_batched(const __grid_constant__ BatchParams B, const int32_t* __restrict__ bfp,
                      const short2* __restrict__ pix, const CandCoef* __restrict__ coef,
                      const float2* __restrict__ ek, const double* __restrict__ gscale,
                      unsigned* qctr) {
  extern __shared__ unsigned char smem_raw[];
  float2* skk = reinterpret_cast<float2*>(smem_raw);  // [P_bf] (kx, ky)
  int* sp = reinterpret_cast<int*>(skk + B.P_bf);     // [P_bf] kept-pixel index
  for (int q = threadIdx.x; q < B.P_bf; q += blockDim.x) {
    const int p = bfp[q];
    const short2 k = pix[p];
    skk[q] = make_float2((float)k.x, (float)k.y);
    sp[q] = p;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // warp tasks from a work queue (list lengths differ between tasks); the
  // numbers a warp takes only grow, so the dataset index only moves forward
  auto take = [&]() -> int {
    unsigned v = 0u;
    if (lane == 0) v = atomicAdd(qctr, 1u);
    return (int)__shfl_sync(0xffffffffu, v, 0);
  };
  int si = 0;
  for (int t = take(); t < B.ntask; t = take()) {
    while (si + 1 < B.n_sets && t >= B.s[si + 1].task0) ++si;  // tasks only grow
    const SetDesc& D = B.s[si];
    const CandCoef cf = coef[si];
    const float2* eks = ek + (size_t)si * B.P_pad;
    const float scale = (float)gscale[2 * si + 1];
    const int tl = t - D.task0;
    const int nyw = (D.Ny + 31) >> 5;
    const int mx = tl / nyw;
    const int my0 = (tl - mx * nyw) * 32;
    const int my = my0 + lane;
    const bool active = my < D.Ny;
    const int mys = active ? my : 0;
    const int mmx = (D.Nx - mx) % D.Nx, mmy = (D.Ny - mys) % D.Ny;
    float Kpx, Kpy, Kmx, Kmy;
    kprime(cf, D.kpm_x, D.kpm_y, freq_index(mx, D.Nx), freq_index(mys, D.Ny), Kpx, Kpy);
    kprime(cf, D.kpm_x, D.kpm_y, freq_index(mmx, D.Nx), freq_index(mmy, D.Ny), Kmx, Kmy);
    const bool nyq = (2 * mx == D.Nx) || (2 * mys == D.Ny);
    const bool nyq_warp = (2 * mx == D.Nx) || (D.Ny / 2 >= my0 && D.Ny / 2 < my0 + 32);
    const float2* Gl = D.G + (size_t)mx * B.P_pad * D.Ny + mys;
    float2 SP = make_float2(0.f, 0.f), SM = make_float2(0.f, 0.f);
    int nP = 0, nM = 0;
    auto contrib = [&](float2 g, float Kx, float Ky, float2 kk, int q, float wp) {
      const float qx = kk.x - Kx, qy = kk.y - Ky;
      const float wm = 1.f - wp;
      const float tq = chi_turns(cf, qx, qy);
      const float fr = tq - rintf(tq);
      float sn, cs;
      __sincosf(kTwoPi * fr, &sn, &cs);
      const float2 e = __ldg(eks + sp[q]);
      const float2 ph = make_float2(e.x * cs - e.y * sn, e.x * sn + e.y * cs);
      const float2 term = cmul(g, ph);
      SP = cmadd(SP, term, wp);
      SM = cmadd(SM, term, wm);
    };
    // at scan rotation 0 the dataset's membership lists give each lane its
    // members in ascending q, the order of the loop below: the same terms
    // in the same order, without the set tests
    const bool lists = D.tl_n != nullptr && cf.c == 1.f && cf.s == 0.f;
    if (lists) {
      int n = D.tl_n[tl];
      if (n < 0 || n > D.tl_cap) n = 0;
      const uint32_t* bits = D.tl_bits + (size_t)tl * (D.tl_cap / 32) * 64;
      const uint32_t* qps = D.tl_qp + (size_t)tl * D.tl_cap;
      for (int e0 = 0; e0 < n; e0 += 32) {
        const uint32_t wP = __ldg(bits + 2 * e0 + lane);
        const uint32_t wM = __ldg(bits + 2 * e0 + 32 + lane);
        const uint32_t ql = __ldg(qps + e0 + lane);
        const int m = n - e0 < 32 ? n - e0 : 32;
        for (int s0 = 0; s0 < m; s0 += kBatch) {
          uint32_t xv[kBatch];
#pragma unroll
          for (int i = 0; i < kBatch; ++i) xv[i] = __shfl_sync(0xffffffffu, ql, s0 + i);
          const unsigned mP = (wP >> s0) & 0xffu, mM = (wM >> s0) & 0xffu;
          nP += __popc(mP);
          nM += __popc(mM);
          const unsigned mAny = mP | mM;
          if (mAny == 0u) continue;
          float2 gb[kBatch];
#pragma unroll
          for (int i = 0; i < kBatch; ++i) {
            const int prow = (int)(xv[i] & 0xffffu);
            gb[i] = ((mAny >> i) & 1u) && prow < B.P_pad ? Gl[(size_t)prow * D.Ny]
                                                          : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int i = 0; i < kBatch; ++i) {
            const bool memP = (mP >> i) & 1u, memM = (mM >> i) & 1u;
            if (!(memP || memM)) continue;
            int q = (int)(xv[i] >> 16);
            if (q >= B.P_bf) q = 0;  // a bad entry: its G is 0, so its term is 0
            const float2 kk = skk[q];
            const float2 g = gb[i];
            if (!nyq_warp) {
              const float2 gg = memM ? make_float2(g.x, -g.y) : g;
              contrib(gg, memM ? Kmx : Kpx, memM ? Kmy : Kpy, kk, q, memM ? 0.f : 1.f);
            } else {
              if (memP) contrib(g, Kpx, Kpy, kk, q, 1.f);
              if (memM) contrib(make_float2(g.x, -g.y), Kmx, Kmy, kk, q, 0.f);
            }
          }
        }
      }
    }
    for (int q0 = 0; q0 < (lists ? 0 : B.P_bf); q0 += kBatch) {
      unsigned mP = 0u, mM = 0u;
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        const int q = q0 + i;
        if (q >= B.P_bf) break;
        const float2 kk = skk[q];
        const float dm = dist2(kk.x, kk.y, Kpx, Kpy);
        const float dp = dist2(kk.x, kk.y, -Kpx, -Kpy);
        const bool memP = active && dm < B.k0sq && dp > B.k0sq;
        bool memM;
        if (!nyq) {
          memM = active && dp < B.k0sq && dm > B.k0sq;
        } else {
          const float em = dist2(kk.x, kk.y, Kmx, Kmy);
          const float ep = dist2(kk.x, kk.y, -Kmx, -Kmy);
          memM = active && em < B.k0sq && ep > B.k0sq;
        }
        mP |= (unsigned)memP << i;
        mM |= (unsigned)memM << i;
      }
      nP += __popc(mP);
      nM += __popc(mM);
      const unsigned mAny = mP | mM;
      if (mAny == 0u) continue;
      float2 gb[kBatch];
#pragma unroll
      for (int i = 0; i < kBatch; ++i)
        gb[i] = ((mAny >> i) & 1u) ? Gl[(size_t)sp[q0 + i] * D.Ny] : make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        const bool memP = (mP >> i) & 1u, memM = (mM >> i) & 1u;
        if (!(memP || memM)) continue;
        const int q = q0 + i;
        const float2 kk = skk[q];
        const float2 g = gb[i];
        if (!nyq_warp) {
          const float2 gg = memM ? make_float2(g.x, -g.y) : g;
          contrib(gg, memM ? Kmx : Kpx, memM ? Kmy : Kpy, kk, q, memM ? 0.f : 1.f);
        } else {
          if (memP) contrib(g, Kpx, Kpy, kk, q, 1.f);
          if (memM) contrib(make_float2(g.x, -g.y), Kmx, Kmy, kk, q, 0.f);
        }
      }
    }
    if (!active) continue;
    D.H[(size_t)my * D.nkx + mx] = combine(SP, SM, nP, nM, D.norm, scale);
  }
}

// V_s = sum_b w(b) |H_s(b)|^2 / N_R^2: partial sums (grid kVarBlocks x n_sets)
__global__ void k_variance_partial_batched(const __grid_constant__ BatchParams B, double* part) {
  __shared__ double red[256];
  const SetDesc& D = B.s[blockIdx.y];
  double sum = 0.0;
  const int n = D.Ny * D.nkx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int mx = i % D.nkx;
    const double w = (mx == 0 || 2 * mx == D.Nx) ? 1.0 : 2.0;
    const float2 v = D.H[i];
    sum += w * ((double)v.x * v.x + (double)v.y * v.y);
  }
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_variance_final_batched(const __grid_constant__ BatchParams B,
                                         const double* __restrict__ part, int nblk, double* var) {
  __shared__ double red[128];
  const int c = blockIdx.x;
  double sum = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) sum += part[(size_t)c * nblk + b];
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double NR = (double)B.s[c].Ny * (double)B.s[c].Nx;
  if (threadIdx.x == 0) var[c] = red[0] / (NR * NR);
}

// Fixed-order sum of nblk rows of nv doubles (one block; deterministic).
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

// First stage of a fixed-order sum of n rows of nv doubles: block b adds the
// rows of its contiguous range [b*n/B, (b+1)*n/B), thread i every 256th from
// the range start, then a fixed tree; out[b][j].
constexpr int kRedBlocks = 152;
__global__ void __launch_bounds__(256) k_reduce_rows(const double* __restrict__ in, long long n,
                                                      int nv, double* out) {
  __shared__ double red[256];
  const long long b0 = n * blockIdx.x / gridDim.x, b1 = n * (blockIdx.x + 1) / gridDim.x;
  for (int j = 0; j < nv; ++j) {
    double s = 0.0;
    for (long long r = b0 + threadIdx.x; r < b1; r += 256) s += in[r * nv + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)blockIdx.x * nv + j] = red[0];
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

// Pixel shard: (sum of G(k, 0) over this plan's bright-field pixels, their
// number) and the trotter scale N_R (the Gbar0 division waits for the sum
// over every shard).
__global__ void k_gbar_part(const float2* __restrict__ G, const int32_t* __restrict__ bfp, int P_bf,
                            int Ny, double NR, double* g0_out, double* gscale) {
  __shared__ double red[256];
  double s = 0.0;
  for (int q = threadIdx.x; q < P_bf; q += blockDim.x) s += (double)G[(size_t)bfp[q] * Ny].x;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    g0_out[0] = red[0];
    g0_out[1] = (double)P_bf;
    gscale[0] = 0.0;
    gscale[1] = NR;
  }
}

// H = H_in / Gbar0, Gbar0 = g0[0] / g0[1] (H = 0 when g0[0] is 0)
__global__ void k_scale_spectrum(const float2* __restrict__ Hin, const double* __restrict__ g0,
                                 size_t n, float2* H) {
  const double f = g0[0] != 0.0 ? g0[1] / g0[0] : 0.0;
  const float ff = (float)f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = Hin[i];
    H[i] = make_float2(v.x * ff, v.y * ff);
  }
}

__global__ void k_ascent(double* theta, const double* step, const double* grad) {
  const int j = threadIdx.x;
  if (j < 5) theta[j] += step[j] * grad[j];
}

// Adam ascent on V in scaled parameters x_j = theta_j / scale_j (moments of
// dV/dx_j = dV/dtheta_j scale_j; beta1 0.9, beta2 0.999, eps 1e-12):
// theta_j += scale_j lr_j mhat_j / (sqrt(vhat_j) + eps).  rate = lr[5],
// scale[5]; state = m1[5], m2[5], step count.  lr_j = 0 holds theta_j.
__global__ void k_adam(double* theta, const double* rate, double* state, const double* grad) {
  const int j = threadIdx.x;
  const double t = state[10] + 1.0;
  if (j < 5) {
    const double sc = rate[5 + j];
    const double g = grad[j] * sc;
    const double m1 = 0.9 * state[j] + 0.1 * g;
    const double m2 = 0.999 * state[5 + j] + 0.001 * g * g;
    state[j] = m1;
    state[5 + j] = m2;
    const double mh = m1 / (1.0 - pow(0.9, t));
    const double vh = m2 / (1.0 - pow(0.999, t));
    if (rate[j] != 0.0) theta[j] += sc * rate[j] * mh / (sqrt(vh) + 1e-12);
  }
  __syncthreads();  // every lane has read the old count
  if (j == 0) state[10] = t;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// candidates per pass of the forward kernel: 8 when their phase tables
// (8 x P_bf float2 in shared memory) still leave 2 CTAs per SM, else 4
// (64 candidates at 1024^2: 12.9 ms with 8, 15.0 ms with 4; on the 512^2
// 25 mrad optics, P_bf = 1963: 18.2 ms with 4, 24.2 ms with 8)
constexpr int kNcFwd = 4;
constexpr int kNcFwdWide = 8;

constexpr int kMaxTrotBlocks = 2048;  // largest trotter grid

// One full wave of the persistent grid: SMs x resident blocks per SM (from the
// occupancy calculator), never more blocks than warp tasks need.
int trot_blocks(const eer4d_plan* p, const void* kern, size_t smem, int* resident = nullptr) {
  const int ntask = p->nkx * (((int)p->g.scan_ny + 31) / 32);
  const int need = (ntask + kWarps - 1) / kWarps;
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, smem);
  int cps = occ > 0 ? occ : 1;
  if (p->tune.trotter_ctas_per_sm > 0 && p->tune.trotter_ctas_per_sm < cps)
    cps = p->tune.trotter_ctas_per_sm;
  int b = nsm * cps;
  if (resident) *resident = b;
  if (b > need) b = need;
  if (b > kMaxTrotBlocks) b = kMaxTrotBlocks;
  return b < 1 ? 1 : b;
}

struct Layout {
  size_t coef, ek, gscale, H, partial, vpart, queue, total;
};
Layout layout(const eer4d_plan* p, int n_cand, int mode) {
  Layout L;
  size_t o = 0;
  L.coef = o; o = align256(o + sizeof(CandCoef) * n_cand);
  L.ek = o; o = align256(o + sizeof(float2) * (size_t)n_cand * p->P_pad);
  L.gscale = o; o = align256(o + 2 * sizeof(double));
  const int nh = (mode == TROT_GRAD || mode == TROT_COUNT) ? 0 : n_cand;
  L.H = o; o = align256(o + sizeof(float2) * (size_t)nh * p->g.scan_ny * p->nkx);
  // the gradient modes: one share per (warp task, lane), then the
  // first-stage sums of the final reduction
  size_t npart = 0;
  if (mode == TROT_GRAD || mode == TROT_VARGRAD) {
    const size_t ntask = (size_t)p->nkx * ((p->g.scan_ny + 31) / 32);
    npart = ntask * 32 + kRedBlocks;
  }
  L.partial = o; o = align256(o + sizeof(double) * 5 * npart);
  L.vpart = o; o = align256(o + sizeof(double) * kVarBlocks * (size_t)nh);
  L.queue = o; o = align256(o + sizeof(unsigned) * (size_t)(n_cand > 0 ? n_cand : 1));
  L.total = o;
  return L;
}

template <int NC>
size_t trot_smem(const eer4d_plan* p) {
  return sizeof(float2) * p->P_bf + sizeof(int) * ((p->P_bf + 1) & ~1) +
         sizeof(float2) * (size_t)NC * p->P_bf;
}

// True when the forward kernel with kNcFwdWide candidates per pass keeps 2
// resident CTAs per SM (its shared-memory tables grow with the candidates).
bool fwd_wide_fits(const eer4d_plan* p) {
  const void* kern = (const void*)k_trotter<TROT_FWD, kNcFwdWide>;
  const size_t sm = trot_smem<kNcFwdWide>(p);
  if (ensure_smem(kern, sm) != cudaSuccess) return false;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, sm) != cudaSuccess)
    return false;
  return occ >= 2;
}

template <int MODE, int NC>
cudaError_t launch_k(const eer4d_plan* p, const TrotParams& tp, const float2* G,
                     const CandCoef* coef, const float2* ek, const double* gsc, const float2* W,
                     float2* H, double* partial, int32_t* count, unsigned* qctr, int* nblk,
                     cudaStream_t s, uint32_t* st) {
  const size_t sm = trot_smem<NC>(p);
  const void* kern = (const void*)k_trotter<MODE, NC>;
  cudaError_t e = ensure_smem(kern, sm);
  if (e != cudaSuccess) return e;
  int resident = 0;
  *nblk = trot_blocks(p, kern, sm, &resident);
  // several forward passes of NC candidates: residency that one pass's warp
  // tasks leave idle takes whole passes (small scans: 64 candidates at 32^2
  // 10.2 -> 1.4 ms, at 256^2 5.6 -> 3.8 ms)
  if constexpr (MODE == TROT_FWD && NC > 1) {
    const int npass = (tp.n_cand + NC - 1) / NC;
    int pg = resident / *nblk;
    if (pg > npass) pg = npass;
    if (pg > 1) {
      const void* ks = (const void*)k_trotter<MODE, NC, true>;
      if ((e = ensure_smem(ks, sm)) != cudaSuccess) return e;
      k_trotter<MODE, NC, true><<<dim3(*nblk, pg), kWarps * 32, sm, s>>>(
          tp, G, p->d_bfp, p->d_pix, coef, ek, gsc, W, H, partial, count, p->d_tl_bits, p->d_tl_qp,
          p->d_tl_n, p->d_tl_order, p->tl_cap, qctr, st);
      return cudaGetLastError();
    }
  }
  k_trotter<MODE, NC><<<*nblk, kWarps * 32, sm, s>>>(tp, G, p->d_bfp, p->d_pix, coef, ek, gsc, W,
                                                     H, partial, count, p->d_tl_bits, p->d_tl_qp,
                                                     p->d_tl_n, p->d_tl_order, p->tl_cap, qctr, st);
  return cudaGetLastError();
}

TrotParams trot_params(const eer4d_plan* p, int n_cand) {
  TrotParams tp;
  tp.Ny = p->g.scan_ny; tp.Nx = p->g.scan_nx; tp.nkx = p->nkx; tp.P_pad = p->P_pad;
  tp.P_bf = p->P_bf;
  tp.kpm_x = (float)p->g.kpm_x; tp.kpm_y = (float)p->g.kpm_y;
  tp.k0sq = (float)(p->g.k0_px * p->g.k0_px);
  tp.norm = p->norm; tp.n_cand = n_cand; tp.NR = (float)p->F;
  return tp;
}

// variance (nullable) and the C2R phase image (nullable) of H [nc][Ny][nkx]
cudaError_t image_stage(const eer4d_plan* p, const float2* H, int nc, double* vpart,
                        float* phase_out, double* var_out, cudaStream_t s) {
  cudaError_t e;
  stage_begin(p, EER4D_STAGE_IMAGE, s);
  if (var_out) {
    k_variance_partial<<<dim3(kVarBlocks, nc), 256, 0, s>>>(H, p->g.scan_ny, p->nkx, p->g.scan_nx,
                                                             vpart);
    k_variance_final<<<nc, 128, 0, s>>>(vpart, kVarBlocks, (double)p->F, var_out);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (phase_out && (e = launch_c2r_image(p, const_cast<float2*>(H), phase_out, nc, s)) != cudaSuccess)
    return e;
  stage_end(p, EER4D_STAGE_IMAGE, s);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_ascent(double* theta, const double* step, const double* grad, cudaStream_t s) {
  k_ascent<<<1, 32, 0, s>>>(theta, step, grad);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_adam(double* theta, const double* rate, double* state, const double* grad,
                        cudaStream_t s) {
  k_adam<<<1, 32, 0, s>>>(theta, rate, state, grad);
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
  unsigned* qctr = reinterpret_cast<unsigned*>(sb + L.queue);
  cudaError_t e;
  stage_begin(p, EER4D_STAGE_TROTTER, s);
  k_prep<<<n_cand, 256, 0, s>>>(aberr, n_cand, p->d_pix, p->P_pad, p->P, p->g.dalpha_rad,
                                p->g.lambda_A, coef, ek, st, 0, qctr);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (mode != TROT_COUNT) {
    k_gbar<<<1, 256, 0, s>>>(G, p->d_bfp, p->P_bf, (int)p->g.scan_ny, (double)p->F, gsc);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const TrotParams tp = trot_params(p, n_cand);
  int nblk = 1;
  switch (mode) {
    case TROT_FWD:
      e = n_cand == 1
              ? launch_k<TROT_FWD, 1>(p, tp, G, coef, ek, gsc, W, H, partial, count_out, qctr, &nblk, s, st)
          : fwd_wide_fits(p)
              ? launch_k<TROT_FWD, kNcFwdWide>(p, tp, G, coef, ek, gsc, W, H, partial, count_out, qctr,
                                               &nblk, s, st)
              : launch_k<TROT_FWD, kNcFwd>(p, tp, G, coef, ek, gsc, W, H, partial, count_out, qctr, &nblk, s, st);
      break;
    case TROT_GRAD:
      e = launch_k<TROT_GRAD, 1>(p, tp, G, coef, ek, gsc, W, H, partial, count_out, qctr, &nblk, s, st);
      break;
    case TROT_VARGRAD:
      e = launch_k<TROT_VARGRAD, 1>(p, tp, G, coef, ek, gsc, W, H, partial, count_out, qctr, &nblk, s, st);
      break;
    default:
      e = launch_k<TROT_COUNT, 1>(p, tp, G, coef, ek, gsc, W, H, partial, count_out, qctr, &nblk, s, st);
      break;
  }
  count_launches(1);
  if (e != cudaSuccess) return e;
  if (mode == TROT_GRAD || mode == TROT_VARGRAD) {
    // the (task, lane) shares in a fixed order: contiguous ranges, then the
    // range sums
    const long long rows = (long long)p->nkx * (((int)p->g.scan_ny + 31) / 32) * 32;
    double* stage = partial + rows * 5;
    k_reduce_rows<<<kRedBlocks, 256, 0, s>>>(partial, rows, 5, stage);
    k_reduce_partials<<<1, 256, 0, s>>>(stage, kRedBlocks, 5, grad_out);
    count_launches(1);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  stage_end(p, EER4D_STAGE_TROTTER, s);
  if (mode == TROT_COUNT || mode == TROT_GRAD) return cudaSuccess;
  return image_stage(p, H, mode == TROT_FWD ? n_cand : 1, vpart, phase_out, var_out, s);
}

cudaError_t launch_trotter_partial(const eer4d_plan* p, const float2* G, const double* aberr,
                                   int n_cand, void* scratch, float2* H_out, double* g0_out,
                                   uint32_t* st, cudaStream_t s) {
  const Layout L = layout(p, n_cand, TROT_FWD);
  unsigned char* sb = static_cast<unsigned char*>(scratch);
  CandCoef* coef = reinterpret_cast<CandCoef*>(sb + L.coef);
  float2* ek = reinterpret_cast<float2*>(sb + L.ek);
  double* gsc = reinterpret_cast<double*>(sb + L.gscale);
  double* partial = reinterpret_cast<double*>(sb + L.partial);
  unsigned* qctr = reinterpret_cast<unsigned*>(sb + L.queue);
  cudaError_t e;
  stage_begin(p, EER4D_STAGE_TROTTER, s);
  k_prep<<<n_cand, 256, 0, s>>>(aberr, n_cand, p->d_pix, p->P_pad, p->P, p->g.dalpha_rad,
                                p->g.lambda_A, coef, ek, st, 0, qctr);
  k_gbar_part<<<1, 256, 0, s>>>(G, p->d_bfp, p->P_bf, (int)p->g.scan_ny, (double)p->F, g0_out, gsc);
  count_launches(2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const TrotParams tp = trot_params(p, n_cand);
  int nblk = 1;
  e = n_cand == 1   ? launch_k<TROT_FWD, 1>(p, tp, G, coef, ek, gsc, nullptr, H_out, partial, nullptr,
                                            qctr, &nblk, s, st)
      : fwd_wide_fits(p) ? launch_k<TROT_FWD, kNcFwdWide>(p, tp, G, coef, ek, gsc, nullptr, H_out,
                                                         partial, nullptr, qctr, &nblk, s, st)
                         : launch_k<TROT_FWD, kNcFwd>(p, tp, G, coef, ek, gsc, nullptr, H_out, partial,
                                                      nullptr, qctr, &nblk, s, st);
  count_launches(1);
  if (e != cudaSuccess) return e;
  stage_end(p, EER4D_STAGE_TROTTER, s);
  return cudaSuccess;
}

cudaError_t launch_image_from_spectrum(const eer4d_plan* p, const float2* H_in, const double* g0,
                                       int n_cand, void* scratch, float* phase_out, double* var_out,
                                       cudaStream_t s) {
  const Layout L = layout(p, n_cand, TROT_FWD);
  unsigned char* sb = static_cast<unsigned char*>(scratch);
  float2* H = reinterpret_cast<float2*>(sb + L.H);
  double* vpart = reinterpret_cast<double*>(sb + L.vpart);
  const size_t n = (size_t)n_cand * p->g.scan_ny * p->nkx;
  k_scale_spectrum<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(H_in, g0, n, H);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return image_stage(p, H, n_cand, vpart, phase_out, var_out, s);
}

namespace {
struct BatchedLayout {
  size_t coef, ek, gscale, vpart, queue, H[kMaxSets], total;
};
BatchedLayout batched_layout(const eer4d_plan* const* plans, int n) {
  BatchedLayout L;
  const eer4d_plan* p0 = plans[0];
  size_t o = 0;
  L.coef = o; o = align256(o + sizeof(CandCoef) * n);
  L.ek = o; o = align256(o + sizeof(float2) * (size_t)n * p0->P_pad);
  L.gscale = o; o = align256(o + 2 * sizeof(double) * n);
  L.vpart = o; o = align256(o + sizeof(double) * kVarBlocks * (size_t)n);
  L.queue = o; o = align256(o + sizeof(unsigned) * (size_t)n);
  for (int i = 0; i < n; ++i) {
    L.H[i] = o;
    o = align256(o + sizeof(float2) * (size_t)plans[i]->g.scan_ny * plans[i]->nkx);
  }
  L.total = o;
  return L;
}
}  // namespace

size_t trotter_batched_scratch_bytes(const eer4d_plan* const* plans, int n) {
  return batched_layout(plans, n).total;
}

cudaError_t launch_trotter_batched(const eer4d_plan* const* plans, const float2* const* G, int n,
                                   const double* aberr, void* scratch, float* const* phase,
                                   double* var, uint32_t* st, cudaStream_t s) {
  const eer4d_plan* p0 = plans[0];
  const BatchedLayout L = batched_layout(plans, n);
  unsigned char* sb = static_cast<unsigned char*>(scratch);
  CandCoef* coef = reinterpret_cast<CandCoef*>(sb + L.coef);
  float2* ek = reinterpret_cast<float2*>(sb + L.ek);
  double* gsc = reinterpret_cast<double*>(sb + L.gscale);
  double* vpart = reinterpret_cast<double*>(sb + L.vpart);
  unsigned* qctr = reinterpret_cast<unsigned*>(sb + L.queue);
  BatchParams B;
  B.n_sets = n;
  B.P_pad = p0->P_pad;
  B.P_bf = p0->P_bf;
  B.k0sq = (float)(p0->g.k0_px * p0->g.k0_px);
  int ntask = 0;
  for (int i = 0; i < kMaxSets; ++i) {
    SetDesc& D = B.s[i];
    if (i >= n) {
      D = B.s[0];
      continue;
    }
    const eer4d_plan* p = plans[i];
    D.G = G[i];
    D.H = reinterpret_cast<float2*>(sb + L.H[i]);
    D.Ny = p->g.scan_ny;
    D.Nx = p->g.scan_nx;
    D.nkx = p->nkx;
    D.norm = p->norm;
    D.kpm_x = (float)p->g.kpm_x;
    D.kpm_y = (float)p->g.kpm_y;
    D.task0 = ntask;
    D.NR = (float)p->F;
    D.tl_bits = p->d_tl_bits;
    D.tl_qp = p->d_tl_qp;
    D.tl_n = p->d_tl_n;
    D.tl_cap = p->tl_cap;
    ntask += p->nkx * ((D.Ny + 31) / 32);
  }
  B.ntask = ntask;
  cudaError_t e;
  stage_begin(p0, EER4D_STAGE_TROTTER, s);
  k_prep<<<n, 256, 0, s>>>(aberr, n, p0->d_pix, p0->P_pad, p0->P, p0->g.dalpha_rad, p0->g.lambda_A,
                           coef, ek, st, 1, qctr);
  k_gbar_batched<<<n, 256, 0, s>>>(B, p0->d_bfp, gsc);
  count_launches(2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t sm = sizeof(float2) * p0->P_bf + sizeof(int) * ((p0->P_bf + 1) & ~1);
  const void* kern = (const void*)k_trotter_batched;
  if ((e = ensure_smem(kern, sm)) != cudaSuccess) return e;
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, sm);
  int nblk = nsm * (occ > 0 ? occ : 1);
  const int need = (ntask + kWarps - 1) / kWarps;
  if (nblk > need) nblk = need;
  if (nblk < 1) nblk = 1;
  k_trotter_batched<<<nblk, kWarps * 32, sm, s>>>(B, p0->d_bfp, p0->d_pix, coef, ek, gsc, qctr);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  stage_end(p0, EER4D_STAGE_TROTTER, s);
  stage_begin(p0, EER4D_STAGE_IMAGE, s);
  if (var) {
    k_variance_partial_batched<<<dim3(kVarBlocks, n), 256, 0, s>>>(B, vpart);
    k_variance_final_batched<<<n, 128, 0, s>>>(B, vpart, kVarBlocks, var);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (phase) {
    for (int i = 0; i < n; ++i) {
      if (!phase[i]) continue;
      if ((e = launch_c2r_image(plans[i], B.s[i].H, phase[i], 1, s)) != cudaSuccess) return e;
    }
  }
  stage_end(p0, EER4D_STAGE_IMAGE, s);
  return cudaSuccess;
}

// ---- membership lists at scan rotation 0 (built once per plan) --------------
// For every warp task (32 consecutive stored bins) the bright-field pixels with
// a member among the task's bins, in ascending q, decided by the same
// member_bits() the trotter kernel runs.  Entry e of task t is
// qp[t][e] = q << 16 | p (bright-field index, kept pixel), and for each chunk
// of 32 entries lane l of the task owns two words, bits[t][chunk][0][l] and
// bits[t][chunk][1][l], whose bit i says whether bin my0 + l is a member of
// K(K'(b)) / K(K'(-b)) through entry 32 chunk + i.  The trotter kernel then
// walks only these pixels when the scan rotation is 0 (mask evaluation is
// about half of its work).
namespace {
__global__ void __launch_bounds__(256) k_trot_lists(int Ny, int Nx, int nkx, int P_bf,
                                                    float kpm_x, float kpm_y, float k0sq,
                                                    const int32_t* __restrict__ bfp,
                                                    const short2* __restrict__ pix,
                                                    uint32_t* bits, uint32_t* qp, int* nlist,
                                                    int cap) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int nyw = (Ny + 31) >> 5;
  if (t >= nkx * nyw) return;  // whole warp
  CandCoef c0;
  c0.c = 1.f;
  c0.s = 0.f;
  const int mx = t / nyw;
  const int my0 = (t - mx * nyw) * 32;
  const int my = my0 + lane;
  const bool active = my < Ny;
  const int mys = active ? my : 0;
  const int mmx = (Nx - mx) % Nx, mmy = (Ny - mys) % Ny;
  float Kpx, Kpy, Kmx, Kmy;
  kprime(c0, kpm_x, kpm_y, freq_index(mx, Nx), freq_index(mys, Ny), Kpx, Kpy);
  kprime(c0, kpm_x, kpm_y, freq_index(mmx, Nx), freq_index(mmy, Ny), Kmx, Kmy);
  const bool nyq = (2 * mx == Nx) || (2 * mys == Ny);
  uint32_t* tb = bits + (size_t)t * (cap / 32) * 64;
  uint32_t* tq = qp + (size_t)t * cap;
  int n = 0;
  uint32_t wP = 0u, wM = 0u;
  for (int q = 0; q < P_bf; ++q) {  // same trip count on every lane
    const int p = bfp[q];
    const short2 k = pix[p];
    bool memP, memM;
    member_bits(make_float2((float)k.x, (float)k.y), Kpx, Kpy, Kmx, Kmy, nyq, active, k0sq, memP,
                memM);
    const unsigned bp = __ballot_sync(0xffffffffu, memP);
    const unsigned bm = __ballot_sync(0xffffffffu, memM);
    if ((bp | bm) != 0u) {  // warp-uniform
      wP |= (uint32_t)memP << (n & 31);
      wM |= (uint32_t)memM << (n & 31);
      if (lane == 0) tq[n] = (uint32_t)q << 16 | (uint32_t)p;
      if ((n & 31) == 31) {
        tb[2 * (n & ~31) + lane] = wP;
        tb[2 * (n & ~31) + 32 + lane] = wM;
        wP = wM = 0u;
      }
      ++n;
    }
  }
  if (n & 31) {
    tb[2 * (n & ~31) + lane] = wP;
    tb[2 * (n & ~31) + 32 + lane] = wM;
  }
  if (lane == 0) nlist[t] = n;
}
}  // namespace

static size_t lists_cap(const eer4d_plan* p) { return ((size_t)p->P_bf + 31) / 32 * 32; }

size_t trotter_lists_bytes(const eer4d_plan* p) {
  const size_t tasks = (size_t)p->nkx * ((p->g.scan_ny + 31) / 32);
  return tasks * lists_cap(p) * (2 * sizeof(uint32_t) + sizeof(uint32_t)) + 2 * tasks * sizeof(int);
}

cudaError_t build_trotter_lists(eer4d_plan* p) {
  const size_t tasks = (size_t)p->nkx * ((p->g.scan_ny + 31) / 32);
  const size_t cap = lists_cap(p);
  if (p->P_pad > 65535) return cudaErrorInvalidValue;  // (q, p) packed in 16 bits each
  cudaError_t e;
  if ((e = cudaMalloc(&p->d_tl_bits, tasks * cap * 2 * sizeof(uint32_t))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&p->d_tl_qp, tasks * cap * sizeof(uint32_t))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&p->d_tl_n, tasks * sizeof(int))) != cudaSuccess) return e;
  // entries past a task's count are never used (their bits are 0); zero them anyway
  if ((e = cudaMemset(p->d_tl_qp, 0, tasks * cap * sizeof(uint32_t))) != cudaSuccess) return e;
  p->tl_cap = (int)cap;
  k_trot_lists<<<(unsigned)((tasks + 7) / 8), 256>>>(
      (int)p->g.scan_ny, (int)p->g.scan_nx, p->nkx, p->P_bf, (float)p->g.kpm_x, (float)p->g.kpm_y,
      (float)(p->g.k0_px * p->g.k0_px), p->d_bfp, p->d_pix, p->d_tl_bits, p->d_tl_qp, p->d_tl_n,
      (int)cap);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(0)) != cudaSuccess) return e;
  // work-queue order: longest lists first (a task's time grows with its list),
  // so the last tasks handed out are short and the warps finish together
  std::vector<int> n(tasks), order(tasks);
  if ((e = cudaMemcpy(n.data(), p->d_tl_n, tasks * sizeof(int), cudaMemcpyDeviceToHost)) !=
      cudaSuccess)
    return e;
  for (size_t i = 0; i < tasks; ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  if ((e = cudaMalloc(&p->d_tl_order, tasks * sizeof(int))) != cudaSuccess) return e;
  return cudaMemcpy(p->d_tl_order, order.data(), tasks * sizeof(int), cudaMemcpyHostToDevice);
}
