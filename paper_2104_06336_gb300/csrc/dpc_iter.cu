// Iterative regularised DPC (Sec. V): gradient descent on ||grad phi / 2 pi - C||
// with the Fourier preconditioner 1/(lam1 + K^2 + lam2 K^4) and step mu, the
// residual taken only over the scan.  As printed the update has no residual
// term; it is read as
//   R = M (C - grad phi^l / 2 pi),
//   phi^{l+1} = phi^l + mu IFFT[ -i (Kx R^x(K) + Ky R^y(K)) / (lam1 + K^2 + lam2 K^4) ],
// phi^0 = 0, on a periodic grid of pad x the scan (pad = 1 or 2; with pad = 2
// the scan sits in the top-left quarter, M = 1 there and 0 in the padding, so
// the solution does not wrap around).  The spectral derivative is iK and the
// update's DC and Nyquist bins (m = M/2 on either axis) are zero, so phi stays
// real.  With pad = 1 and lam1 = lam2 = 0 the iteration reaches the one-shot
// Fourier integration as (1 - (1 - mu)^L).
//
// phi is kept as its spectrum Phi; each step is one inverse transform of
// (iKx + i iKy) Phi (the two real gradients packed as one complex field), the
// residual, one forward transform (the two real residuals packed) and the
// update of Phi.
#include "common.cuh"

namespace {

__device__ __forceinline__ bool nyq_bin(int m, int M) { return 2 * m == M; }

__global__ void k_dpc_setup(const float* __restrict__ com, int Ny, int Nx, int My, int Mx,
                            float cscale, float2* Cpk, float2* Phi) {
  const size_t n = (size_t)My * Mx;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / Mx), x = (int)(i - (size_t)y * Mx);
    float2 c = make_float2(0.f, 0.f);
    if (y < Ny && x < Nx) {
      const size_t f = (size_t)y * Nx + x;
      c = make_float2(com[f] * cscale, com[(size_t)Ny * Nx + f] * cscale);
    }
    Cpk[i] = c;
    Phi[i] = make_float2(0.f, 0.f);
  }
}

// Z = (i Kx + i (i Ky)) Phi = Phi (-Ky + i Kx), zero at Nyquist bins
__global__ void k_dpc_deriv(const float2* __restrict__ Phi, int My, int Mx, float inv_lx,
                            float inv_ly, float2* Z) {
  const size_t n = (size_t)My * Mx;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int my = (int)(i / Mx), mx = (int)(i - (size_t)my * Mx);
    float2 z = make_float2(0.f, 0.f);
    if (!nyq_bin(mx, Mx) && !nyq_bin(my, My)) {
      const float kx = freq_index(mx, Mx) * inv_lx, ky = freq_index(my, My) * inv_ly;
      const float2 p = Phi[i];
      z = make_float2(-ky * p.x - kx * p.y, -ky * p.y + kx * p.x);
    }
    Z[i] = z;
  }
}

// Z = M (C - g) with g = Z (packed gradients), M = 1 on the scan
__global__ void k_dpc_resid(const float2* __restrict__ Cpk, int Ny, int Nx, int My, int Mx,
                            float2* Z) {
  const size_t n = (size_t)My * Mx;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / Mx), x = (int)(i - (size_t)y * Mx);
    const float2 c = Cpk[i], g = Z[i];
    Z[i] = (y < Ny && x < Nx) ? make_float2(c.x - g.x, c.y - g.y) : make_float2(0.f, 0.f);
  }
}

// Phi(K) += mu * (-i (Kx Rx + Ky Ry) / den), Rx = (Z(K) + conj Z(-K))/2,
// Ry = -i (Z(K) - conj Z(-K))/2; DC and Nyquist bins unchanged.  One thread
// per pair {K, -K}.
__device__ __forceinline__ float2 update_one(float2 z, float2 zm, float kx, float ky, float lam1,
                                             float lam2) {
  const float2 X = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
  const float2 Y = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
  const float k2 = kx * kx + ky * ky;
  const float den = lam1 + k2 + lam2 * k2 * k2;
  if (den == 0.f) return make_float2(0.f, 0.f);
  const float2 s = make_float2(kx * X.x + ky * Y.x, kx * X.y + ky * Y.y);
  return make_float2(s.y / den, -s.x / den);
}

__global__ void k_dpc_update(const float2* __restrict__ Z, int My, int Mx, float inv_lx,
                             float inv_ly, float lam1, float lam2, float mu, float2* Phi) {
  const size_t n = (size_t)My * Mx;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int my = (int)(i / Mx), mx = (int)(i - (size_t)my * Mx);
    const int mmy = (My - my) % My, mmx = (Mx - mx) % Mx;
    const size_t im = (size_t)mmy * Mx + mmx;
    if (im < i) continue;  // the partner handles the pair
    if (i == 0 || nyq_bin(mx, Mx) || nyq_bin(my, My)) continue;
    const float2 z = Z[i], zm = Z[im];
    const float kx = freq_index(mx, Mx) * inv_lx, ky = freq_index(my, My) * inv_ly;
    const float kxm = freq_index(mmx, Mx) * inv_lx, kym = freq_index(mmy, My) * inv_ly;
    const float2 u = update_one(z, zm, kx, ky, lam1, lam2);
    const float2 um = update_one(zm, z, kxm, kym, lam1, lam2);
    float2 p = Phi[i];
    Phi[i] = make_float2(p.x + mu * u.x, p.y + mu * u.y);
    if (im != i) {
      p = Phi[im];
      Phi[im] = make_float2(p.x + mu * um.x, p.y + mu * um.y);
    }
  }
}

__global__ void k_dpc_out(const float2* __restrict__ Z, int Ny, int Nx, int Mx, float* phase) {
  const size_t n = (size_t)Ny * Nx;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / Nx), x = (int)(i - (size_t)y * Nx);
    phase[i] = Z[(size_t)y * Mx + x].x;
  }
}

unsigned grid_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? b : 4096);
}

}  // namespace

size_t dpc_iterative_scratch_bytes(const eer4d_plan* p, int pad) {
  return 3 * sizeof(float2) * (size_t)pad * pad * p->F;
}

cudaError_t launch_dpc_iterative(const eer4d_plan* p, const float* com, double lam1, double lam2,
                                 double mu, int n_iter, int pad, void* scratch, float* phase,
                                 cudaStream_t s) {
  const int Ny = p->g.scan_ny, Nx = p->g.scan_nx;
  const FftDesc& fy = pad == 2 ? p->fy2 : p->fy;
  const FftDesc& fx = pad == 2 ? p->fx2 : p->fx;
  const int My = fy.N, Mx = fx.N;
  const size_t n = (size_t)My * Mx;
  float2* Phi = static_cast<float2*>(scratch);
  float2* Z = Phi + n;
  float2* Cpk = Z + n;
  const float cscale = (float)(p->g.dalpha_raw_rad / p->g.lambda_A);
  const float inv_lx = (float)(1.0 / ((double)Mx * p->g.step_A));
  const float inv_ly = (float)(1.0 / ((double)My * p->g.step_A));
  const unsigned gb = grid_for(n);
  stage_begin(p, EER4D_STAGE_DPC, s);
  k_dpc_setup<<<gb, 256, 0, s>>>(com, Ny, Nx, My, Mx, cscale, Cpk, Phi);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  const float inv_n = 1.f / ((float)My * (float)Mx);
  for (int l = 0; l < n_iter && e == cudaSuccess; ++l) {
    k_dpc_deriv<<<gb, 256, 0, s>>>(Phi, My, Mx, inv_lx, inv_ly, Z);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = launch_fft2_c2c(fy, fx, Z, -1, inv_n, s)) != cudaSuccess) break;
    k_dpc_resid<<<gb, 256, 0, s>>>(Cpk, Ny, Nx, My, Mx, Z);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = launch_fft2_c2c(fy, fx, Z, 1, 1.f, s)) != cudaSuccess) break;
    k_dpc_update<<<gb, 256, 0, s>>>(Z, My, Mx, inv_lx, inv_ly, (float)lam1, (float)lam2, (float)mu,
                                    Phi);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(Z, Phi, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return e;
  if ((e = launch_fft2_c2c(fy, fx, Z, -1, inv_n, s)) != cudaSuccess) return e;
  k_dpc_out<<<grid_for((size_t)Ny * Nx), 256, 0, s>>>(Z, Ny, Nx, Mx, phase);
  count_launches(1);
  stage_end(p, EER4D_STAGE_DPC, s);
  return cudaGetLastError();
}
