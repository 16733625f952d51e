// G-function viewer (Fig. 2, middle panel: G(k, K) at a few selected scan
// frequencies K, used to judge the residual aberrations by eye).  A gather
// from the resident G: for each requested bin (m_y, m_x) the kept pixels'
// values are placed on the binned detector window, zero elsewhere.  G is
// stored for K_x >= 0; the other half is read as G(k, -K) = conj G(k, K).
#include "common.cuh"

namespace {

struct Bins {
  int my[EER4D_MAX_SLICES], mx[EER4D_MAX_SLICES];
};

__global__ void k_g_slices(const float2* __restrict__ G, Bins B, const short2* __restrict__ pix,
                           int P, int P_pad, int Ny, int Nx, int pw, int ph, int dc_u, int dc_v,
                           float2* out) {
  const int s = blockIdx.y;
  const int my = B.my[s], mx = B.mx[s];
  const bool flip = 2 * mx > Nx;  // not stored: use the conjugate at -K
  const int sx = flip ? (Nx - mx) % Nx : mx;
  const int sy = flip ? (Ny - my) % Ny : my;
  float2* o = out + (size_t)s * pw * ph;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pw * ph; i += gridDim.x * blockDim.x)
    o[i] = make_float2(0.f, 0.f);
  __syncthreads();  // one block per slice: its zero fill ends before its scatter
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const short2 k = pix[p];
    float2 g = G[((size_t)sx * P_pad + p) * Ny + sy];
    if (flip) g.y = -g.y;
    o[(size_t)(k.y + dc_v) * pw + (k.x + dc_u)] = g;
  }
}

}  // namespace

cudaError_t launch_g_slices(const eer4d_plan* p, const float2* G, const int32_t* bins, int n,
                            float2* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  Bins B;
  for (int i = 0; i < EER4D_MAX_SLICES; ++i) {
    B.my[i] = i < n ? bins[2 * i] : 0;
    B.mx[i] = i < n ? bins[2 * i + 1] : 0;
  }
  k_g_slices<<<dim3(1, n), 256, 0, s>>>(G, B, p->d_pix, p->P, p->P_pad, (int)p->g.scan_ny,
                                        (int)p->g.scan_nx, (int)p->g.pw, (int)p->g.ph,
                                        (int)p->g.dc_u, (int)p->g.dc_v, out);
  count_launches(1);
  return cudaGetLastError();
}
