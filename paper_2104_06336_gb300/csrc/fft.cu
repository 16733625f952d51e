// Scan-axis transforms: the G function (Sec. IV, G(k,K) = F_{R->K} I(k,R)),
// the inverse transform of the SSB spectrum to the phase image, the forward
// transform of an upstream phase gradient, and the Fourier integration of the
// COM field (Sec. V).  All are batched Stockham FFTs in shared memory
// (fft.cuh); real data use the two-real-rows-in-one-complex-transform form.
#include "fft.cuh"
#include "fft_reg.cuh"

namespace {

constexpr int kThreads = 256;

// Column transforms of a [N][ld] complex array (element n of column c at
// n*ld + c), nb columns per CTA, batch = blockIdx.y.
__global__ void __launch_bounds__(kThreads) k_fft_cols(const float2* in, float2* out, FftDesc d,
                                                       int dir, int ncols, int ld_in, int ld_out,
                                                       long long bs_in, long long bs_out, int nb,
                                                       float scale) {
  extern __shared__ float2 sm[];
  const int N = d.N;
  float2* A = sm;
  float2* B = sm + (size_t)nb * N;
  const int c0 = blockIdx.x * nb;
  in += blockIdx.y * bs_in;
  out += blockIdx.y * bs_out;
  const int tot = N * nb;
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    const int n = w / nb, b = w - n * nb, c = c0 + b;
    A[w] = c < ncols ? in[(size_t)n * ld_in + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* res = fft_smem(A, B, d, dir, nb, 1, nb, true);
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    const int n = w / nb, b = w - n * nb, c = c0 + b;
    if (c < ncols) out[(size_t)n * ld_out + c] = cscale(res[w], scale);
  }
}

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

// Real rows -> half spectra (k = 0..N/2).  Row (a, c) starts at a*in_sa +
// c*in_sc; its spectrum value k goes to k*out_skx + a*out_sa + c*out_sc.  A CTA
// takes TA consecutive rows a0..a0+TA-1 (TA even) at c = blockIdx.y + c0 and
// transforms pairs z = row_2b + i row_2b+1; A = (Z(k) + conj Z(-k))/2,
// B = -i (Z(k) - conj Z(-k))/2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_rows_r2c(const T* in, float2* out, FftDesc d,
                                                       int nA, int TA, int c0, long long in_sa,
                                                       long long in_sc, long long out_skx,
                                                       long long out_sa, long long out_sc,
                                                       int a_fast) {
  extern __shared__ float2 sm[];
  const int N = d.N, nb = TA / 2;
  float2* A = sm;
  float2* B = sm + (size_t)nb * N;
  const int a0 = blockIdx.x * TA;
  const int c = c0 + blockIdx.y;
  float* Af = reinterpret_cast<float*>(A);
  const int tot = TA * N;
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    const int al = w / N, n = w - al * N, a = a0 + al;
    float v = a < nA ? to_f<T>(in[a * in_sa + c * in_sc + n]) : 0.f;
    Af[2 * ((al >> 1) * N + n) + (al & 1)] = v;
  }
  __syncthreads();
  const float2* res = fft_smem(A, B, d, 1, nb, N, 1, false);
  const int nk = N / 2 + 1;
  const int tot2 = TA * nk;
  for (int w = threadIdx.x; w < tot2; w += blockDim.x) {
    int al, k;
    if (a_fast) { al = w % TA; k = w / TA; } else { k = w % nk; al = w / nk; }
    const int a = a0 + al;
    if (a >= nA) continue;
    const int b = al >> 1;
    const float2 z = res[b * N + k];
    const float2 zm = res[b * N + (k == 0 ? 0 : N - k)];
    float2 v;
    if ((al & 1) == 0) v = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    else v = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    out[k * out_skx + a * out_sa + c * out_sc] = v;
  }
}

// Half spectra -> real rows (inverse).  Row (a, c) value k (0..N/2) is read at
// c*in_sc + a*in_sa + k; the real output row at c*out_sc + a*out_sa.  The
// imaginary parts of k = 0 and k = N/2 are ignored.  Output scaled by scale.
__global__ void __launch_bounds__(kThreads) k_rows_c2r(const float2* in, float* out, FftDesc d,
                                                       int nA, int TA, long long in_sa,
                                                       long long in_sc, long long out_sa,
                                                       long long out_sc, float scale) {
  extern __shared__ float2 sm[];
  const int N = d.N, nb = TA / 2, h = N / 2;
  float2* A = sm;
  float2* B = sm + (size_t)nb * N;
  const int a0 = blockIdx.x * TA;
  const int c = blockIdx.y;
  in += c * in_sc;
  out += c * out_sc;
  const int tot = nb * N;
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    const int b = w / N, k = w - b * N;
    const int ra = a0 + 2 * b, rb = ra + 1;
    const int kk = k <= h ? k : N - k;
    float2 x = ra < nA ? in[ra * in_sa + kk] : make_float2(0.f, 0.f);
    float2 y = rb < nA ? in[rb * in_sa + kk] : make_float2(0.f, 0.f);
    if (kk == 0 || kk == h) { x.y = 0.f; y.y = 0.f; }
    if (k > h) { x.y = -x.y; y.y = -y.y; }
    A[w] = make_float2(x.x - y.y, x.y + y.x);
  }
  __syncthreads();
  const float2* res = fft_smem(A, B, d, -1, nb, N, 1, false);
  const int tot2 = TA * N;
  for (int w = threadIdx.x; w < tot2; w += blockDim.x) {
    const int al = w / N, n = w - al * N, a = a0 + al;
    if (a >= nA) continue;
    const float2 z = res[(al >> 1) * N + n];
    out[a * out_sa + n] = ((al & 1) ? z.y : z.x) * scale;
  }
}

// Complex rows [rows][N] in place; with real_out, writes Re(x)*scale to
// real_out instead.
__global__ void __launch_bounds__(kThreads) k_rows_c2c(float2* data, float* real_out, FftDesc d,
                                                       int rows, int nb, int dir, float scale) {
  extern __shared__ float2 sm[];
  const int N = d.N;
  float2* A = sm;
  float2* B = sm + (size_t)nb * N;
  const int r0 = blockIdx.x * nb;
  const int tot = nb * N;
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    const int b = w / N, n = w - b * N;
    A[w] = r0 + b < rows ? data[(size_t)(r0 + b) * N + n] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* res = fft_smem(A, B, d, dir, nb, N, 1, false);
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    const int b = w / N, n = w - b * N;
    if (r0 + b >= rows) continue;
    if (real_out) real_out[(size_t)(r0 + b) * N + n] = res[w].x * scale;
    else data[(size_t)(r0 + b) * N + n] = cscale(res[w], scale);
  }
}

// Fourier integration of the COM field (Sec. V), in place on Z = F(Cx + i Cy):
// X = F(Cx) = (Z(K) + conj Z(-K))/2, Y = F(Cy) = -i (Z(K) - conj Z(-K))/2,
// Phi(K) = -i (Kx X + Ky Y) / (lam1 + K^2 + lam2 K^4), Phi(0) = 0.
// One thread per bin pair {K, -K}.
__device__ __forceinline__ float2 idpc_one(float2 z, float2 zm, float kx, float ky, float lam1,
                                           float lam2) {
  const float2 X = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
  const float2 Y = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
  const float k2 = kx * kx + ky * ky;
  const float den = lam1 + k2 + lam2 * k2 * k2;
  if (den == 0.f) return make_float2(0.f, 0.f);
  const float2 s = make_float2(kx * X.x + ky * Y.x, kx * X.y + ky * Y.y);
  return make_float2(s.y / den, -s.x / den);  // -i s / den
}

__global__ void k_idpc_filter(float2* Z, int Ny, int Nx, float inv_lx, float inv_ly, float lam1,
                              float lam2) {
  const int F = Ny * Nx;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x) {
    const int my = f / Nx, mx = f - my * Nx;
    const int mmy = (Ny - my) % Ny, mmx = (Nx - mx) % Nx;
    const int fm = mmy * Nx + mmx;
    if (fm < f) continue;  // the partner thread handles this pair
    const float2 z = Z[f], zm = Z[fm];
    const float kx = freq_index(mx, Nx) * inv_lx, ky = freq_index(my, Ny) * inv_ly;
    const float kxm = freq_index(mmx, Nx) * inv_lx, kym = freq_index(mmy, Ny) * inv_ly;
    float2 p = idpc_one(z, zm, kx, ky, lam1, lam2);
    float2 pm = idpc_one(zm, z, kxm, kym, lam1, lam2);
    if (f == 0) p = make_float2(0.f, 0.f);
    Z[f] = p;
    if (fm != f) Z[fm] = pm;
  }
}

// out[b][c][r] = in[b][r][c] for a batch of [rows][cols] complex matrices
__global__ void k_transpose(const float2* __restrict__ in, float2* __restrict__ out, int rows,
                            int cols) {
  __shared__ float2 t[32][33];
  const size_t b = blockIdx.z;
  in += b * (size_t)rows * cols;
  out += b * (size_t)rows * cols;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(size_t)c * rows + r] = t[threadIdx.x][i];
  }
}

int cols_nb(int N) {
  int nb = 16;
  while (nb > 1 && (size_t)2 * nb * N * sizeof(float2) > 96 * 1024) nb >>= 1;
  return nb;
}
int rows_nb(int N) {  // complex transforms per CTA for row kernels
  int nb = 8;
  while (nb > 1 && (size_t)2 * nb * N * sizeof(float2) > 96 * 1024) nb >>= 1;
  return nb;
}

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
  return ensure_smem((const void*)kern, bytes);
}

cudaError_t cols(const FftDesc& d, const float2* in, float2* out, int dir, int ncols, int ld_in,
                 int ld_out, long long bs_in, long long bs_out, int nbatch, float scale,
                 cudaStream_t s) {
  const int nb = cols_nb(d.N);
  const size_t sm = (size_t)2 * nb * d.N * sizeof(float2);
  cudaError_t e = set_smem(k_fft_cols, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((ncols + nb - 1) / nb, nbatch);
  k_fft_cols<<<grid, kThreads, sm, s>>>(in, out, d, dir, ncols, ld_in, ld_out, bs_in, bs_out, nb,
                                        scale);
  count_launches(1);
  return cudaGetLastError();
}

// ---- register four-step dispatch (power-of-two N in [16, 1024]) ----------
bool reg_size(int N) { return N >= 16 && N <= 1024 && (N & (N - 1)) == 0; }

template <int R1, int R2, int CB, int DIR, bool TOUT>
cudaError_t cols_reg_t(const FftDesc& d, const float2* in, float2* out, int ncols, int ld_in,
                       int ld_out, long long bs_in, long long bs_out, int nbatch, float scale,
                       cudaStream_t s) {
  constexpr int NT = (R1 > R2 ? R1 : R2) * CB;
  const size_t sm = sizeof(float2) * ((size_t)R1 * CB * (R2 + 1) + 2 * CB);
  auto kern = k_colfft_reg<R1, R2, CB, DIR, TOUT>;
  cudaError_t e = set_smem(kern, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((ncols + CB - 1) / CB, nbatch);
  if (!d.tw4 || reg_r1(d.N) != R1) return cudaErrorInvalidValue;
  kern<<<grid, NT, sm, s>>>(in, out, d.tw4, ncols, ld_in, ld_out, bs_in, bs_out, scale);
  count_launches(1);
  return cudaGetLastError();
}

template <int DIR, bool TOUT = false>
cudaError_t cols_reg(const FftDesc& d, const float2* in, float2* out, int ncols, int ld_in,
                     int ld_out, long long bs_in, long long bs_out, int nbatch, float scale,
                     cudaStream_t s) {
#define EER4D_COLS(R1, R2, CB) \
  return cols_reg_t<R1, R2, CB, DIR, TOUT>(d, in, out, ncols, ld_in, ld_out, bs_in, bs_out, nbatch, scale, s)
  switch (d.N) {
    case 1024: EER4D_COLS(32, 32, 8);
    case 512: EER4D_COLS(32, 16, 8);
    case 256: EER4D_COLS(16, 16, 16);
    case 128: EER4D_COLS(16, 8, 16);
    case 64: EER4D_COLS(8, 8, 32);
    case 32: EER4D_COLS(8, 4, 32);
    default: EER4D_COLS(4, 4, 64);
  }
#undef EER4D_COLS
}

template <int R1, int R2, int CP>
cudaError_t r2c_reg_t(const FftDesc& d, const __half* in, float2* out, int nA, int c0, int nc,
                      long long in_sa, long long in_sc, long long out_skx, long long out_sa,
                      long long out_sc, cudaStream_t s) {
  constexpr int N = R1 * R2;
  const size_t a = (size_t)R1 * CP * (R2 + 1), b = (size_t)N * CP;
  const size_t sm = sizeof(float2) * (a > b ? a : b);
  auto kern = k_rowfft_r2c_reg<R1, R2, CP>;
  cudaError_t e = set_smem(kern, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((nA + 2 * CP - 1) / (2 * CP), nc);
  if (!d.tw4 || reg_r1(d.N) != R1) return cudaErrorInvalidValue;
  kern<<<grid, R1 * CP, sm, s>>>(in, out, d.tw4, nA, c0, in_sa, in_sc, out_skx, out_sa, out_sc);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t r2c_reg(const FftDesc& d, const __half* in, float2* out, int nA, int c0, int nc,
                    long long in_sa, long long in_sc, long long out_skx, long long out_sa,
                    long long out_sc, cudaStream_t s) {
#define EER4D_R2C(R1, R2, CP) \
  return r2c_reg_t<R1, R2, CP>(d, in, out, nA, c0, nc, in_sa, in_sc, out_skx, out_sa, out_sc, s)
  switch (d.N) {
    case 1024: EER4D_R2C(32, 32, 8);
    case 512: EER4D_R2C(32, 16, 8);
    case 256: EER4D_R2C(16, 16, 16);
    case 128: EER4D_R2C(16, 8, 16);
    case 64: EER4D_R2C(8, 8, 32);
    case 32: EER4D_R2C(8, 4, 32);
    default: EER4D_R2C(4, 4, 64);
  }
#undef EER4D_R2C
}

}  // namespace

cudaError_t launch_transpose(const float2* in, float2* out, int rows, int cols, int batch,
                             cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch);
  k_transpose<<<grid, dim3(32, 8), 0, s>>>(in, out, rows, cols);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_stage1(const eer4d_plan* p, const __half* counts, float2* G, int y0, int y1,
                          cudaStream_t s) {
  if (y1 <= y0) return cudaSuccess;
  const FftDesc& d = p->fx;
  const long long NRl = p->cstride;
  if (reg_size(d.N) && p->precision != EER4D_FP32_STOCKHAM) {
    stage_begin(p, EER4D_STAGE_DFT_X, s);
    cudaError_t e = r2c_reg(d, counts, G, p->P_pad, y0, y1 - y0, NRl, (long long)p->g.scan_nx,
                            (long long)p->g.scan_ny * p->P_pad, 1, (long long)p->P_pad, s);
    stage_end(p, EER4D_STAGE_DFT_X, s);
    return e;
  }
  const int nb = rows_nb(d.N);
  const int TA = 2 * nb;
  const size_t sm = (size_t)2 * nb * d.N * sizeof(float2);
  cudaError_t e = set_smem(k_rows_r2c<__half>, sm);
  if (e != cudaSuccess) return e;
  const long long NR = p->cstride;
  dim3 grid((p->P_pad + TA - 1) / TA, y1 - y0);
  stage_begin(p, EER4D_STAGE_DFT_X, s);
  k_rows_r2c<__half><<<grid, kThreads, sm, s>>>(
      counts, G, d, p->P_pad, TA, y0, NR, (long long)p->g.scan_nx,
      (long long)p->g.scan_ny * p->P_pad, 1, (long long)p->P_pad, 1);
  count_launches(1);
  stage_end(p, EER4D_STAGE_DFT_X, s);
  return cudaGetLastError();
}

cudaError_t launch_stage2(const eer4d_plan* p, const float2* X1, float2* G, cudaStream_t s) {
  const int Ny = p->g.scan_ny;
  const long long bs = (long long)Ny * p->P_pad;
  stage_begin(p, EER4D_STAGE_DFT_Y, s);
  cudaError_t e;
  if (reg_size(p->fy.N) && p->precision != EER4D_FP32_STOCKHAM) {
    e = cols_reg<1, true>(p->fy, X1, G, p->P_pad, p->P_pad, Ny, bs, bs, p->nkx, 1.f, s);
  } else {
    // generic lengths: in-place column FFT, then a tiled transpose into G
    e = cols(p->fy, X1, const_cast<float2*>(X1), 1, p->P_pad, p->P_pad, p->P_pad, bs, bs, p->nkx,
             1.f, s);
    if (e == cudaSuccess) e = launch_transpose(X1, G, Ny, p->P_pad, p->nkx, s);
  }
  stage_end(p, EER4D_STAGE_DFT_Y, s);
  return e;
}

cudaError_t launch_c2r_image(const eer4d_plan* p, float2* H, float* phase, int n_cand,
                             cudaStream_t s) {
  const int Ny = p->g.scan_ny, Nx = p->g.scan_nx, nkx = p->nkx;
  const long long bs = (long long)Ny * nkx;
  cudaError_t e = reg_size(p->fy.N) ? cols_reg<-1>(p->fy, H, H, nkx, nkx, nkx, bs, bs, n_cand, 1.f, s)
                                    : cols(p->fy, H, H, -1, nkx, nkx, nkx, bs, bs, n_cand, 1.f, s);
  if (e != cudaSuccess) return e;
  const FftDesc& d = p->fx;
  const int nb = rows_nb(d.N), TA = 2 * nb;
  const size_t sm = (size_t)2 * nb * d.N * sizeof(float2);
  e = set_smem(k_rows_c2r, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((Ny + TA - 1) / TA, n_cand);
  k_rows_c2r<<<grid, kThreads, sm, s>>>(H, phase, d, Ny, TA, nkx, bs, Nx, (long long)Ny * Nx,
                                        1.f / ((float)Ny * (float)Nx));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_r2c_image(const eer4d_plan* p, const float* g, float2* W, cudaStream_t s) {
  const int Ny = p->g.scan_ny, Nx = p->g.scan_nx, nkx = p->nkx;
  const FftDesc& d = p->fx;
  const int nb = rows_nb(d.N), TA = 2 * nb;
  const size_t sm = (size_t)2 * nb * d.N * sizeof(float2);
  cudaError_t e = set_smem(k_rows_r2c<float>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((Ny + TA - 1) / TA, 1);
  k_rows_r2c<float><<<grid, kThreads, sm, s>>>(g, W, d, Ny, TA, 0, Nx, 0, 1, nkx, 0, 0);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long bs = (long long)Ny * nkx;
  return cols(p->fy, W, W, 1, nkx, nkx, nkx, bs, bs, 1, 1.f, s);
}

template <int R1, int R2, int CB, int DIR, bool REAL_OUT>
cudaError_t rows_reg_t(const FftDesc& d, float2* data, float* real_out, int rows, float scale,
                       cudaStream_t s) {
  constexpr int NT = (R1 > R2 ? R1 : R2) * CB;
  const size_t sm = sizeof(float2) * (size_t)CB * R1 * (R2 + 1);
  auto kern = k_rowfft_c2c_reg<R1, R2, CB, DIR, REAL_OUT>;
  cudaError_t e = set_smem(kern, sm);
  if (e != cudaSuccess) return e;
  if (!d.tw4 || reg_r1(d.N) != R1) return cudaErrorInvalidValue;
  kern<<<(rows + CB - 1) / CB, NT, sm, s>>>(data, real_out, d.tw4, rows, d.N, scale);
  count_launches(1);
  return cudaGetLastError();
}

// Register four-step transform of every row of [rows][d.N] in place (or its
// real part times scale into real_out); d.N a register length (reg_size).
template <int DIR, bool REAL_OUT = false>
cudaError_t rows_reg(const FftDesc& d, float2* data, float* real_out, int rows, float scale,
                     cudaStream_t s) {
#define EER4D_ROWS(R1, R2, CB) return rows_reg_t<R1, R2, CB, DIR, REAL_OUT>(d, data, real_out, rows, scale, s)
  switch (d.N) {
    case 1024: EER4D_ROWS(32, 32, 4);
    case 512: EER4D_ROWS(32, 16, 4);
    case 256: EER4D_ROWS(16, 16, 8);
    case 128: EER4D_ROWS(16, 8, 8);
    case 64: EER4D_ROWS(8, 8, 16);
    case 32: EER4D_ROWS(8, 4, 16);
    default: EER4D_ROWS(4, 4, 32);
  }
#undef EER4D_ROWS
}

cudaError_t launch_fft2_c2c(const FftDesc& fy, const FftDesc& fx, float2* data, int dir,
                            float scale, cudaStream_t s) {
  const int My = fy.N, Mx = fx.N;
  if (reg_size(Mx) && reg_size(My)) {
    cudaError_t e = dir > 0 ? rows_reg<1>(fx, data, nullptr, My, 1.f, s)
                            : rows_reg<-1>(fx, data, nullptr, My, 1.f, s);
    if (e != cudaSuccess) return e;
    return dir > 0 ? cols_reg<1>(fy, data, data, Mx, Mx, Mx, 0, 0, 1, scale, s)
                   : cols_reg<-1>(fy, data, data, Mx, Mx, Mx, 0, 0, 1, scale, s);
  }
  const int nb = rows_nb(Mx);
  const size_t sm = (size_t)2 * nb * Mx * sizeof(float2);
  cudaError_t e = set_smem(k_rows_c2c, sm);
  if (e != cudaSuccess) return e;
  k_rows_c2c<<<(My + nb - 1) / nb, kThreads, sm, s>>>(data, nullptr, fx, My, nb, dir, 1.f);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cols(fy, data, data, dir, Mx, Mx, Mx, 0, 0, 1, scale, s);
}

cudaError_t launch_idpc(const eer4d_plan* p, float2* z, float* phase, double lam1, double lam2,
                        cudaStream_t s) {
  const int Ny = p->g.scan_ny, Nx = p->g.scan_nx;
  const FftDesc& dx = p->fx;
  const int nb = rows_nb(dx.N);
  const size_t sm = (size_t)2 * nb * dx.N * sizeof(float2);
  cudaError_t e = set_smem(k_rows_c2c, sm);
  if (e != cudaSuccess) return e;
  stage_begin(p, EER4D_STAGE_DPC, s);
  const float inv_lx = (float)(1.0 / ((double)Nx * p->g.step_A));
  const float inv_ly = (float)(1.0 / ((double)Ny * p->g.step_A));
  if (reg_size(Nx) && reg_size(Ny)) {
    // register four-step tiles: rows, columns (in place), filter, columns, rows
    if ((e = rows_reg<1>(dx, z, nullptr, Ny, 1.f, s)) != cudaSuccess) return e;
    if ((e = cols_reg<1>(p->fy, z, z, Nx, Nx, Nx, 0, 0, 1, 1.f, s)) != cudaSuccess) return e;
    k_idpc_filter<<<(Ny * Nx + 255) / 256, 256, 0, s>>>(z, Ny, Nx, inv_lx, inv_ly, (float)lam1,
                                                         (float)lam2);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cols_reg<-1>(p->fy, z, z, Nx, Nx, Nx, 0, 0, 1, 1.f, s)) != cudaSuccess) return e;
    e = rows_reg<-1, true>(dx, z, phase, Ny, 1.f / ((float)Ny * (float)Nx), s);
    stage_end(p, EER4D_STAGE_DPC, s);
    return e;
  }
  k_rows_c2c<<<(Ny + nb - 1) / nb, kThreads, sm, s>>>(z, nullptr, dx, Ny, nb, 1, 1.f);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cols(p->fy, z, z, 1, Nx, Nx, Nx, 0, 0, 1, 1.f, s)) != cudaSuccess) return e;
  k_idpc_filter<<<(Ny * Nx + 255) / 256, 256, 0, s>>>(z, Ny, Nx, inv_lx, inv_ly, (float)lam1,
                                                       (float)lam2);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cols(p->fy, z, z, -1, Nx, Nx, Nx, 0, 0, 1, 1.f, s)) != cudaSuccess) return e;
  k_rows_c2c<<<(Ny + nb - 1) / nb, kThreads, sm, s>>>(z, phase, dx, Ny, nb, -1,
                                                       1.f / ((float)Ny * (float)Nx));
  count_launches(1);
  stage_end(p, EER4D_STAGE_DPC, s);
  return cudaGetLastError();
}
