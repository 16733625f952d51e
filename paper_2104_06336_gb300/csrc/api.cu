// C ABI of libeer4d: plan construction and the entry points declared in
// include/eer4d.h.  Host code only validates arguments, derives launch
// parameters and enqueues kernels; every step of the path runs on the GPU.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "common.cuh"

#include <atomic>
#include <mutex>
#include <map>
#include <utility>

namespace {

thread_local char g_last_error[256] = "";
std::atomic<unsigned long long> g_launches{0};

int cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return EER4D_OK;
  snprintf(g_last_error, sizeof g_last_error, "%s", cudaGetErrorString(e));
  return EER4D_ECUDA;
}

int factorize(int N, int* radix) {
  int n = N, k = 0;
  while (n % 8 == 0) { radix[k++] = 8; n /= 8; }
  while (n % 4 == 0) { radix[k++] = 4; n /= 4; }
  while (n % 2 == 0) { radix[k++] = 2; n /= 2; }
  for (int p = 3; n > 1; p += 2) {
    while (n % p == 0) {
      if (k >= EER4D_MAX_STAGES) return -1;
      radix[k++] = p;
      n /= p;
    }
  }
  return k;
}

// twiddles exp(-2 pi i j / N) from the exact integer j, in double
cudaError_t make_fft(int N, FftDesc& d, float2** dev) {
  d.N = N;
  d.nst = factorize(N, d.radix);
  if (d.nst < 0) return cudaErrorInvalidValue;
  const int r1 = reg_r1(N), r2 = r1 ? N / r1 : 0;
  std::vector<float2> tw(r1 ? 2 * N : N);
  const double tp = 6.283185307179586476925286766559;
  for (int j = 0; j < N; ++j) {
    tw[j] = make_float2((float)cos(tp * j / N), (float)-sin(tp * j / N));
  }
  for (int k1 = 0; k1 < r1; ++k1)
    for (int j2 = 0; j2 < r2; ++j2) tw[N + k1 * r2 + j2] = tw[j2 * k1];  // j2 k1 < N
  cudaError_t e = cudaMalloc(dev, sizeof(float2) * tw.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(*dev, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
  d.tw = *dev;
  d.tw4 = r1 ? *dev + N : nullptr;
  return e;
}

template <typename T>
cudaError_t upload(T** dev, const std::vector<T>& h) {
  cudaError_t e = cudaMalloc(dev, sizeof(T) * (h.empty() ? 1 : h.size()));
  if (e != cudaSuccess) return e;
  if (h.empty()) return cudaSuccess;
  return cudaMemcpy(*dev, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

bool geom_ok(const eer4d_geom* g) {
  if (!g) return false;
  if (g->det_w == 0 || g->det_h == 0 || (uint64_t)g->det_w * g->det_h > 0xFFFFFFFFull) return false;
  if (g->det_w > 32767 || g->det_h > 32767) return false;
  if (g->bin == 0 || g->pw == 0 || g->ph == 0 || g->dc_u >= g->pw || g->dc_v >= g->ph) return false;
  if (g->pw > 32767 || g->ph > 32767) return false;
  if (!(g->k0_px > 0.0) || !(g->crop_px >= g->k0_px)) return false;
  if (g->scan_ny < 2 || g->scan_nx < 2 || g->scan_ny > 4096 || g->scan_nx > 4096) return false;
  if ((g->scan_ny & 1) || (g->scan_nx & 1)) return false;
  if (!(g->kpm_x > 0.0) || !(g->kpm_y > 0.0) || !(g->lambda_A > 0.0) || !(g->dalpha_rad > 0.0)) return false;
  if (!(g->step_A > 0.0) || !(g->dalpha_raw_rad > 0.0)) return false;
  return true;
}

void free_plan(eer4d_plan* p) {
  if (!p) return;
  cudaFree(p->d_lutx);
  cudaFree(p->d_luty);
  cudaFree(p->d_lut2);
  cudaFree(p->d_lutp);
  cudaFree(p->d_pix);
  cudaFree(p->d_bfp);
  cudaFree(p->d_rows);
  cudaFree(p->d_tl_bits);
  cudaFree(p->d_tl_qp);
  cudaFree(p->d_tl_n);
  cudaFree(p->d_tl_order);
  cudaFree(p->d_tw_y);
  cudaFree(p->d_tw_x);
  cudaFree(p->d_tw_y2);
  cudaFree(p->d_tw_x2);
  cudaFree(p->d_dft_hi);
  cudaFree(p->d_dft_lo);
  cudaFree(p->d_tc4_tabs);
  cudaFree(p->d_tc4_tw);
  free(p);
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t kTrotterListsMaxBytes = (size_t)512 << 20;

}  // namespace

int cuda_status(cudaError_t e) { return cuda_fail(e); }

size_t work_counts_bytes(const eer4d_plan* p) { return (size_t)2 * p->P_pad * p->cstride; }
size_t work_bytes(const eer4d_plan* p) {
  if (dft2_fused_ok(p)) return al256(work_counts_bytes(p)) + al256(dft2_ring_bytes(p)) + dft2_ctl_bytes(p);
  return al256(work_counts_bytes(p)) + sizeof(float2) * (size_t)p->nkx * p->g.scan_ny * p->P_pad;
}

void stage_begin(const eer4d_plan* p, int stage, cudaStream_t s) {
  if (p && p->ev_start[stage]) cudaEventRecord(p->ev_start[stage], s);
}
void stage_end(const eer4d_plan* p, int stage, cudaStream_t s) {
  if (p && p->ev_stop[stage]) cudaEventRecord(p->ev_stop[stage], s);
}
cudaError_t ensure_smem(const void* kernel, size_t bytes) {
  // the opt-in covers dynamic + static shared memory above 48 KB, so it is set
  // for every sizeable dynamic request (static arrays of up to 16 KB beside it)
  if (bytes <= 32 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;  // (kernel, device) -> bytes set
  std::lock_guard<std::mutex> lk(mu);
  int dev = 0;
  cudaGetDevice(&dev);
  const std::pair<const void*, int> key(kernel, dev);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[key] = bytes;
  return e;
}

void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

extern "C" {

uint64_t eer4d_launch_count(void) { return g_launches.load(); }

int eer4d_set_stage_events(eer4d_plan* p, void* const* ev_start, void* const* ev_stop) {
  if (!p) return EER4D_EINVAL;
  for (int i = 0; i < EER4D_N_STAGES; ++i) {
    p->ev_start[i] = ev_start ? static_cast<cudaEvent_t>(ev_start[i]) : nullptr;
    p->ev_stop[i] = ev_stop ? static_cast<cudaEvent_t>(ev_stop[i]) : nullptr;
  }
  return EER4D_OK;
}

const char* eer4d_last_error(void) { return g_last_error; }

int eer4d_shard_range(int P, int shard, int n_shards, int* h_begin, int* h_end) {
  if (P < 1 || n_shards < 1 || n_shards > EER4D_MAX_SHARDS || shard < 0 || shard >= n_shards ||
      !h_begin || !h_end)
    return EER4D_EINVAL;
  *h_begin = (int)((long long)P * shard / n_shards);
  *h_end = (int)((long long)P * (shard + 1) / n_shards);
  return EER4D_OK;
}

static int create_plan(const eer4d_geom* h_geom, int precision, int norm, int shard, int n_shards,
                       eer4d_plan** out);

int eer4d_plan_create(const eer4d_geom* h_geom, int precision, int norm, eer4d_plan** out) {
  return create_plan(h_geom, precision, norm, 0, 1, out);
}

int eer4d_plan_create_shard(const eer4d_geom* h_geom, int precision, int norm, int shard,
                            int n_shards, eer4d_plan** out) {
  if (n_shards < 1 || n_shards > EER4D_MAX_SHARDS || shard < 0 || shard >= n_shards)
    return EER4D_EINVAL;
  return create_plan(h_geom, precision, norm, shard, n_shards, out);
}

static int create_plan(const eer4d_geom* h_geom, int precision, int norm, int shard, int n_shards,
                       eer4d_plan** out) {
  if (!out) return EER4D_EINVAL;
  *out = nullptr;
  if (!geom_ok(h_geom)) return EER4D_EINVAL;
  if (precision != EER4D_FP32_FFT && precision != EER4D_SPLIT_FP16 &&
      precision != EER4D_FP32_FFT_2PASS && precision != EER4D_FP32_STOCKHAM)
    return EER4D_EINVAL;
  if (norm != EER4D_NORM_NONE && norm != EER4D_NORM_AREA) return EER4D_EINVAL;
  const eer4d_geom& g = *h_geom;
  eer4d_plan* p = static_cast<eer4d_plan*>(calloc(1, sizeof(eer4d_plan)));
  if (!p) return EER4D_ENOMEM;
  p->g = g;
  p->precision = precision;
  p->norm = norm;
  p->F = (int)(g.scan_ny * g.scan_nx);
#ifndef EER4D_COUNTS_PAD
#define EER4D_COUNTS_PAD 0
#endif
  p->cstride = (long long)p->F + EER4D_COUNTS_PAD;
  p->nkx = (int)g.scan_nx / 2 + 1;
  p->dw.init(g.det_w);

  // kept pixels (|k| < crop, double) numbered row-major; bright-field
  // |k|^2 < k0^2 in float32.  A shard plan keeps the range [p_begin, p_end)
  // of that numbering, renumbered from 0.
  const double crop2 = g.crop_px * g.crop_px;
  int P_all = 0;
  for (uint32_t v = 0; v < g.ph; ++v)
    for (uint32_t u = 0; u < g.pw; ++u) {
      const int kx = (int)u - (int)g.dc_u, ky = (int)v - (int)g.dc_v;
      if ((double)(kx * kx + ky * ky) < crop2) ++P_all;
    }
  if (P_all == 0) { free_plan(p); return EER4D_EINVAL; }
  if (eer4d_shard_range(P_all, shard, n_shards, &p->p_begin, &p->p_end) != EER4D_OK ||
      p->p_end <= p->p_begin) {
    free_plan(p);
    return EER4D_EINVAL;
  }
  p->shard = shard;
  p->n_shards = n_shards;
  std::vector<int32_t> lut2((size_t)g.pw * g.ph, -1);
  std::vector<short2> pix;
  std::vector<int4> rows;
  const float k0sq = (float)(g.k0_px * g.k0_px);
  int P_bf = 0, gi = -1;
  for (uint32_t v = 0; v < g.ph; ++v) {
    const int ky = (int)v - (int)g.dc_v;
    int lo = 1, hi = 0, plo = -1;
    for (uint32_t u = 0; u < g.pw; ++u) {
      const int kx = (int)u - (int)g.dc_u;
      if ((double)(kx * kx + ky * ky) < crop2 && ++gi >= p->p_begin && gi < p->p_end) {
        const int idx = (int)pix.size();
        lut2[(size_t)v * g.pw + u] = idx;
        pix.push_back(make_short2((short)kx, (short)ky));
        if ((float)(kx * kx + ky * ky) < k0sq) {
          if (lo > hi) {
            lo = hi = kx;
            plo = idx;
          } else {
            if (kx != hi + 1) { free_plan(p); return EER4D_EINVAL; }  // BF row not contiguous
            hi = kx;
          }
          ++P_bf;
        }
      }
    }
    if (lo <= hi) rows.push_back(make_int4(ky, lo, hi, plo));
  }
  p->P = (int)pix.size();
  if (p->P == 0 || p->P > 32767 || P_bf == 0) { free_plan(p); return EER4D_EINVAL; }
  p->P_bf = P_bf;
  p->P_pad = (p->P + 15) / 16 * 16;
  p->n_rows = (int)rows.size();
  p->list_max = (P_bf + 1) & ~1;
  pix.resize(p->P_pad, make_short2(0, 0));
  std::vector<int32_t> bfp;  // kept-pixel index of every bright-field pixel, row-major
  for (const int4& R : rows)
    for (int kx = R.y; kx <= R.z; ++kx) bfp.push_back(R.w + (kx - R.y));

  std::vector<int16_t> lutx(g.det_w), luty(g.det_h);
  for (uint32_t x = 0; x < g.det_w; ++x) {
    const long long d = (long long)x - g.crop_x0;
    const long long u = d >= 0 ? d / g.bin : -1;
    lutx[x] = (int16_t)((d >= 0 && u < (long long)g.pw) ? u : -1);
  }
  for (uint32_t y = 0; y < g.det_h; ++y) {
    const long long d = (long long)y - g.crop_y0;
    const long long v = d >= 0 ? d / g.bin : -1;
    luty[y] = (int16_t)((d >= 0 && v < (long long)g.ph) ? v : -1);
  }
  // raw pixel -> kept pixel in one table (one lookup per event in the scatter)
  std::vector<int16_t> lutp;
  if ((uint64_t)g.det_w * g.det_h <= (1ull << 24)) {
    lutp.assign((size_t)g.det_w * g.det_h, (int16_t)-1);
    for (uint32_t y = 0; y < g.det_h; ++y) {
      if (luty[y] < 0) continue;
      for (uint32_t x = 0; x < g.det_w; ++x) {
        if (lutx[x] < 0) continue;
        lutp[(size_t)y * g.det_w + x] = (int16_t)lut2[(size_t)luty[y] * g.pw + lutx[x]];
      }
    }
  }
  cudaError_t e;
  if (!lutp.empty() && (e = upload(&p->d_lutp, lutp)) != cudaSuccess) {
    const int rc = e == cudaErrorMemoryAllocation ? EER4D_ENOMEM : cuda_fail(e);
    free_plan(p);
    return rc;
  }
  if ((e = upload(&p->d_lutx, lutx)) != cudaSuccess || (e = upload(&p->d_luty, luty)) != cudaSuccess ||
      (e = upload(&p->d_lut2, lut2)) != cudaSuccess || (e = upload(&p->d_pix, pix)) != cudaSuccess ||
      (e = upload(&p->d_bfp, bfp)) != cudaSuccess ||
      (e = upload(&p->d_rows, rows)) != cudaSuccess ||
      (e = make_fft((int)g.scan_ny, p->fy, &p->d_tw_y)) != cudaSuccess ||
      (e = make_fft((int)g.scan_nx, p->fx, &p->d_tw_x)) != cudaSuccess ||
      (e = make_fft(2 * (int)g.scan_ny, p->fy2, &p->d_tw_y2)) != cudaSuccess ||
      (e = make_fft(2 * (int)g.scan_nx, p->fx2, &p->d_tw_x2)) != cudaSuccess) {
    const int rc = e == cudaErrorMemoryAllocation ? EER4D_ENOMEM : cuda_fail(e);
    free_plan(p);
    return rc;
  }
  // trotter membership lists at rotation 0 when they are small enough to keep
  if (trotter_lists_bytes(p) <= kTrotterListsMaxBytes && build_trotter_lists(p) != cudaSuccess) {
    cudaGetLastError();  // lists are optional: without them the kernel evaluates the masks
    cudaFree(p->d_tl_bits);
    cudaFree(p->d_tl_qp);
    cudaFree(p->d_tl_n);
    cudaFree(p->d_tl_order);
    p->d_tl_bits = nullptr;
    p->d_tl_qp = nullptr;
    p->d_tl_n = nullptr;
    p->d_tl_order = nullptr;
  }
  if (precision == EER4D_SPLIT_FP16 && g.scan_nx == 1024 && (e = make_dftx_tc4(p)) != cudaSuccess) {
    const int rc = e == cudaErrorMemoryAllocation ? EER4D_ENOMEM : cuda_fail(e);
    free_plan(p);
    return rc;
  }
  if (precision == EER4D_SPLIT_FP16 && (e = make_dftx_tc(p)) != cudaSuccess) {
    const int rc = e == cudaErrorMemoryAllocation ? EER4D_ENOMEM : cuda_fail(e);
    free_plan(p);
    return rc;
  }
  p->next_frame = 0;
  *out = p;
  return EER4D_OK;
}

void eer4d_plan_destroy(eer4d_plan* plan) { free_plan(plan); }

int eer4d_plan_info(const eer4d_plan* p, eer4d_info* info) {
  if (!p || !info) return EER4D_EINVAL;
  info->P = p->P;
  info->P_pad = p->P_pad;
  info->P_bf = p->P_bf;
  info->n_rows = p->n_rows;
  info->nkx = p->nkx;
  info->trotter_list_max = 2 * p->P_bf;
  info->p_begin = p->p_begin;
  info->p_end = p->p_end;
  return EER4D_OK;
}

int eer4d_workspace_bytes(const eer4d_plan* p, int n_cand, size_t* counts_bytes, size_t* G_bytes,
                          size_t* scratch_bytes) {
  if (!p || n_cand < 1 || n_cand > 1024) return EER4D_EINVAL;
  if (counts_bytes) *counts_bytes = work_bytes(p);
  if (G_bytes) *G_bytes = sizeof(float2) * (size_t)p->nkx * p->g.scan_ny * p->P_pad;
  if (scratch_bytes) {
    size_t s = sizeof(float2) * (size_t)p->F;  // com_dpc
    if (vdet_scratch_bytes(p) > s) s = vdet_scratch_bytes(p);
    size_t r = trotter_scratch_bytes(p, n_cand, TROT_FWD);
    if (r > s) s = r;
    r = trotter_scratch_bytes(p, 1, TROT_GRAD) + sizeof(float2) * (size_t)p->g.scan_ny * p->nkx;
    if (r > s) s = r;
    r = trotter_scratch_bytes(p, 1, TROT_VARGRAD);
    if (r > s) s = r;
    *scratch_bytes = s;
  }
  return EER4D_OK;
}

int eer4d_status_code(const uint32_t* st) {
  if (!st) return EER4D_EINVAL;
  const uint32_t b = st[0];
  if (b & EER4D_ST_OFFSETS) return EER4D_EOFFSETS;
  if (b & EER4D_ST_RANGE) return EER4D_ERANGE;
  if (b & EER4D_ST_OVERFLOW) return EER4D_EOVERFLOW;
  if (b & EER4D_ST_TIMEOUT) return EER4D_ETIMEOUT;
  if (b & EER4D_ST_ROTATION) return EER4D_EINVAL;
  if (b & EER4D_ST_BOUNDS) return EER4D_EBOUNDS;
  return EER4D_OK;
}

const char* eer4d_strerror(int code) {
  switch (code) {
    case EER4D_OK: return "ok";
    case EER4D_EINVAL: return "invalid argument";
    case EER4D_ERANGE: return "event index outside the detector (events dropped)";
    case EER4D_EOFFSETS: return "frame offsets decreasing or beyond the event array";
    case EER4D_EOVERFLOW: return "more than 2048 events in one binned pixel of one frame";
    case EER4D_ETIMEOUT: return "a bounded device wait timed out";
    case EER4D_ECUDA: return "CUDA error";
    case EER4D_ENOMEM: return "out of memory";
    case EER4D_EORDER: return "chunks not delivered in frame order";
    case EER4D_ESCRATCH: return "plan needs more scratch than the 8 MiB static array of ssb_reconstruct_static";
    case EER4D_EBOUNDS: return "a bounds check of the debug build failed (access skipped)";
    default: return "unknown error";
  }
}

int eer_load_csr(const eer4d_plan* p, const uint32_t* d_idx, uint64_t n_idx, const uint64_t* d_off,
                 uint64_t n_frames, int64_t* d_pacbed, int64_t* d_totals, uint32_t* d_status,
                 void* stream) {
  if (!p || !d_off || (n_idx && !d_idx)) return EER4D_EINVAL;
  if (n_frames == 0) return EER4D_OK;
  return cuda_fail(launch_validate(p, d_idx, n_idx, d_off, n_frames, d_pacbed, d_totals, d_status,
                                   (cudaStream_t)stream));
}

int eer_decode_rle(const uint32_t* d_runs, uint64_t n, const uint64_t* d_off, uint64_t n_frames,
                   uint32_t* d_idx, uint32_t* d_status, void* stream) {
  if (!d_off || (n && (!d_runs || !d_idx))) return EER4D_EINVAL;
  return cuda_fail(launch_rle_decode(d_runs, n, d_off, n_frames, d_idx, d_status,
                                     (cudaStream_t)stream));
}

int virtual_detectors(const eer4d_plan* p, const uint32_t* d_idx, uint64_t n_idx,
                      const uint64_t* d_off, uint64_t n_frames, const double* h_radii, int n_rings,
                      const int64_t* d_totals, double cx, double cy, void* d_scratch,
                      int32_t* d_out, uint32_t* d_status, void* stream) {
  if (!p || !d_off || (n_idx && !d_idx) || !h_radii || !d_scratch || !d_out) return EER4D_EINVAL;
  if (n_rings < 1 || n_rings > EER4D_MAX_RINGS) return EER4D_EINVAL;
  for (int j = 0; j <= n_rings; ++j)
    if (!(h_radii[j] >= 0.0) || (j && h_radii[j] < h_radii[j - 1])) return EER4D_EINVAL;
  return cuda_fail(launch_virtual_detectors(p, d_idx, n_idx, d_off, n_frames, h_radii, n_rings,
                                            d_totals, cx, cy, d_scratch, d_out, d_status,
                                            (cudaStream_t)stream));
}

int dpc_iterative(const eer4d_plan* p, const float* d_com, double lam1, double lam2, double mu,
                  int n_iter, int pad, void* d_scratch, size_t scratch_bytes, float* d_phase,
                  void* stream) {
  if (!p || !d_com || !d_scratch || !d_phase) return EER4D_EINVAL;
  if ((pad != 1 && pad != 2) || n_iter < 0 || n_iter > 100000) return EER4D_EINVAL;
  if (!(mu > 0.0 && mu < 2.0) || !(lam1 >= 0.0) || !(lam2 >= 0.0)) return EER4D_EINVAL;
  if (scratch_bytes < dpc_iterative_scratch_bytes(p, pad)) return EER4D_EINVAL;
  return cuda_fail(launch_dpc_iterative(p, d_com, lam1, lam2, mu, n_iter, pad, d_scratch, d_phase,
                                        (cudaStream_t)stream));
}

int com_dpc(const eer4d_plan* p, const uint32_t* d_idx, uint64_t n_idx, const uint64_t* d_off,
            int64_t* d_sums, float* d_com, float* d_phase, const int64_t* d_totals, double cx,
            double cy, double lam1, double lam2, void* d_scratch, uint32_t* d_status, void* stream) {
  if (!p || !d_off || (n_idx && !d_idx) || !d_sums || !d_com) return EER4D_EINVAL;
  if (d_phase && !d_scratch) return EER4D_EINVAL;
  if (!(lam1 >= 0.0) || !(lam2 >= 0.0)) return EER4D_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float2* z = d_phase ? static_cast<float2*>(d_scratch) : nullptr;
  int rc = cuda_fail(launch_com(p, d_idx, n_idx, d_off, d_sums, d_com, z, d_totals, cx, cy,
                                d_status, s));
  if (rc != EER4D_OK || !d_phase) return rc;
  return cuda_fail(launch_idpc(p, z, d_phase, lam1, lam2, s));
}

int com_dpc_sums(const eer4d_plan* p, const int64_t* d_sums, float* d_com, float* d_phase,
                 const int64_t* d_totals, double cx, double cy, double lam1, double lam2,
                 void* d_scratch, uint32_t* d_status, void* stream) {
  (void)d_status;
  if (!p || !d_sums || !d_com) return EER4D_EINVAL;
  if (d_phase && !d_scratch) return EER4D_EINVAL;
  if (!(lam1 >= 0.0) || !(lam2 >= 0.0)) return EER4D_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float2* z = d_phase ? static_cast<float2*>(d_scratch) : nullptr;
  int rc = cuda_fail(launch_com_from_sums(p, d_sums, d_com, z, d_totals, cx, cy, s));
  if (rc != EER4D_OK || !d_phase) return rc;
  return cuda_fail(launch_idpc(p, z, d_phase, lam1, lam2, s));
}

static int accumulate(eer4d_plan* p, const uint32_t* d_idx, uint64_t n_idx, const uint64_t* d_off,
                      uint64_t first_frame, uint64_t n_frames, void* d_counts, void* d_G,
                      int is_last, int64_t* d_sums, int64_t* d_totals, uint32_t* d_status,
                      void* stream) {
  if (!p || !d_off || (n_idx && !d_idx) || !d_counts || !d_G) return EER4D_EINVAL;
  const uint64_t F = (uint64_t)p->F;
  const uint64_t end = first_frame + n_frames;
  if (end > F || end < first_frame) return EER4D_EINVAL;
  if (is_last && end != F) return EER4D_EINVAL;
  if (first_frame == 0) p->next_frame = 0;
  if (first_frame != p->next_frame) return EER4D_EORDER;
  cudaStream_t s = (cudaStream_t)stream;
  __half* counts = static_cast<__half*>(d_counts);
  float2* X1 = reinterpret_cast<float2*>(static_cast<unsigned char*>(d_counts) +
                                         al256(work_counts_bytes(p)));
  float2* G = static_cast<float2*>(d_G);
  int rc = cuda_fail(launch_scatter(p, d_idx, n_idx, d_off, first_frame, n_frames, counts,
                                    d_status, s, d_sums, d_totals));
  if (rc != EER4D_OK) return rc;
  const uint64_t Nx = p->g.scan_nx;
  if (dft2_fused_ok(p)) {  // both axes in one launch once every frame is in
    p->next_frame = end;
    if (is_last) {
      unsigned char* ctl = reinterpret_cast<unsigned char*>(X1) + al256(dft2_ring_bytes(p));
      rc = cuda_fail(launch_dft2_fused(p, counts, X1, G, reinterpret_cast<unsigned*>(ctl),
                                       d_status, s));
      p->next_frame = 0;
    }
    return rc;
  }
  const int ya = (int)(first_frame / Nx), yb = (int)(end / Nx);
  rc = cuda_fail(p->precision == EER4D_SPLIT_FP16
                     ? launch_stage1_tc(p, counts, X1, ya, yb, d_status, s)
                     : launch_stage1(p, counts, X1, ya, yb, s));
  if (rc != EER4D_OK) return rc;
  p->next_frame = end;
  if (is_last) {
    rc = cuda_fail(launch_stage2(p, X1, G, s));
    p->next_frame = 0;
  }
  return rc;
}

int ssb_accumulate(eer4d_plan* p, const uint32_t* d_idx, uint64_t n_idx, const uint64_t* d_off,
                   uint64_t first_frame, uint64_t n_frames, void* d_counts, void* d_G, int is_last,
                   uint32_t* d_status, void* stream) {
  return accumulate(p, d_idx, n_idx, d_off, first_frame, n_frames, d_counts, d_G, is_last, nullptr,
                    nullptr, d_status, stream);
}

int ssb_accumulate_com(eer4d_plan* p, const uint32_t* d_idx, uint64_t n_idx, const uint64_t* d_off,
                       uint64_t first_frame, uint64_t n_frames, void* d_counts, void* d_G,
                       int is_last, int64_t* d_sums, int64_t* d_totals, uint32_t* d_status,
                       void* stream) {
  if (!d_sums || !d_totals) return EER4D_EINVAL;
  return accumulate(p, d_idx, n_idx, d_off, first_frame, n_frames, d_counts, d_G, is_last, d_sums,
                    d_totals, d_status, stream);
}

int ssb_reconstruct(const eer4d_plan* p, const void* d_G, const double* d_aberr, int n_cand,
                    void* d_scratch, float* d_phase, double* d_var, uint32_t* d_status,
                    void* stream) {
  if (!p || !d_G || !d_aberr || !d_scratch || n_cand < 1 || n_cand > 1024) return EER4D_EINVAL;
  return cuda_fail(launch_trotter(p, static_cast<const float2*>(d_G), d_aberr, n_cand, TROT_FWD,
                                  d_scratch, nullptr, d_phase, d_var, nullptr, nullptr, d_status,
                                  (cudaStream_t)stream));
}

int ssb_spectrum_partial(const eer4d_plan* p, const void* d_G, const double* d_aberr, int n_cand,
                         void* d_scratch, void* d_H, double* d_g0, uint32_t* d_status,
                         void* stream) {
  if (!p || !d_G || !d_aberr || !d_scratch || !d_H || !d_g0 || n_cand < 1 || n_cand > 1024)
    return EER4D_EINVAL;
  if (p->norm != EER4D_NORM_NONE) return EER4D_EINVAL;
  return cuda_fail(launch_trotter_partial(p, static_cast<const float2*>(d_G), d_aberr, n_cand,
                                          d_scratch, static_cast<float2*>(d_H), d_g0, d_status,
                                          (cudaStream_t)stream));
}

int ssb_image_from_spectrum(const eer4d_plan* p, const void* d_H, const double* d_g0, int n_cand,
                            void* d_scratch, float* d_phase, double* d_var, void* stream) {
  if (!p || !d_H || !d_g0 || !d_scratch || n_cand < 1 || n_cand > 1024) return EER4D_EINVAL;
  return cuda_fail(launch_image_from_spectrum(p, static_cast<const float2*>(d_H), d_g0, n_cand,
                                              d_scratch, d_phase, d_var, (cudaStream_t)stream));
}

int ssb_grad(const eer4d_plan* p, const void* d_G, const double* d_aberr, const float* d_grad_phase,
             double* d_grad, void* d_scratch, uint32_t* d_status, void* stream) {
  if (!p || !d_G || !d_aberr || !d_grad_phase || !d_grad || !d_scratch) return EER4D_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float2* W = reinterpret_cast<float2*>(static_cast<unsigned char*>(d_scratch) +
                                        trotter_scratch_bytes(p, 1, TROT_GRAD));
  int rc = cuda_fail(launch_r2c_image(p, d_grad_phase, W, s));
  if (rc != EER4D_OK) return rc;
  return cuda_fail(launch_trotter(p, static_cast<const float2*>(d_G), d_aberr, 1, TROT_GRAD,
                                  d_scratch, W, nullptr, nullptr, d_grad, nullptr, d_status, s));
}

int ssb_variance_grad(const eer4d_plan* p, const void* d_G, const double* d_aberr, void* d_scratch,
                      float* d_phase, double* d_var, double* d_grad, uint32_t* d_status,
                      void* stream) {
  if (!p || !d_G || !d_aberr || !d_scratch || !d_var || !d_grad) return EER4D_EINVAL;
  return cuda_fail(launch_trotter(p, static_cast<const float2*>(d_G), d_aberr, 1, TROT_VARGRAD,
                                  d_scratch, nullptr, d_phase, d_var, d_grad, nullptr, d_status,
                                  (cudaStream_t)stream));
}

int ssb_refocus_step(const eer4d_plan* p, const void* d_G, double* d_aberr, const double* d_step,
                     void* d_scratch, float* d_phase, double* d_var, double* d_grad,
                     uint32_t* d_status, void* stream) {
  if (!p || !d_G || !d_aberr || !d_step || !d_scratch || !d_var || !d_grad) return EER4D_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = cuda_fail(launch_trotter(p, static_cast<const float2*>(d_G), d_aberr, 1, TROT_VARGRAD,
                                    d_scratch, nullptr, d_phase, d_var, d_grad, nullptr, d_status, s));
  if (rc != EER4D_OK) return rc;
  return cuda_fail(launch_ascent(d_aberr, d_step, d_grad, s));
}

int ssb_refocus_step_adam(const eer4d_plan* p, const void* d_G, double* d_aberr, const double* d_rate,
                          double* d_state, void* d_scratch, float* d_phase, double* d_var,
                          double* d_grad, uint32_t* d_status, void* stream) {
  if (!p || !d_G || !d_aberr || !d_rate || !d_state || !d_scratch || !d_var || !d_grad)
    return EER4D_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = cuda_fail(launch_trotter(p, static_cast<const float2*>(d_G), d_aberr, 1, TROT_VARGRAD,
                                    d_scratch, nullptr, d_phase, d_var, d_grad, nullptr, d_status, s));
  if (rc != EER4D_OK) return rc;
  return cuda_fail(launch_adam(d_aberr, d_rate, d_state, d_grad, s));
}

static bool same_detector(const eer4d_plan* a, const eer4d_plan* b) {
  const eer4d_geom &x = a->g, &y = b->g;
  return x.det_w == y.det_w && x.det_h == y.det_h && x.bin == y.bin && x.crop_x0 == y.crop_x0 &&
         x.crop_y0 == y.crop_y0 && x.pw == y.pw && x.ph == y.ph && x.dc_u == y.dc_u &&
         x.dc_v == y.dc_v && x.k0_px == y.k0_px && x.crop_px == y.crop_px &&
         x.lambda_A == y.lambda_A && x.dalpha_rad == y.dalpha_rad && a->P == b->P &&
         a->P_pad == b->P_pad && a->P_bf == b->P_bf;
}

static int check_batch(const eer4d_plan* const* plans, int n) {
  if (!plans || n < 1 || n > EER4D_MAX_SETS) return EER4D_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!plans[i] || !same_detector(plans[0], plans[i])) return EER4D_EINVAL;
  return EER4D_OK;
}

int eer4d_batched_scratch_bytes(const eer4d_plan* const* plans, int n, size_t* bytes) {
  const int rc = check_batch(plans, n);
  if (rc != EER4D_OK || !bytes) return rc != EER4D_OK ? rc : EER4D_EINVAL;
  *bytes = trotter_batched_scratch_bytes(plans, n);
  return EER4D_OK;
}

int ssb_reconstruct_batched(const eer4d_plan* const* plans, const void* const* d_G, int n,
                            const double* d_aberr, void* d_scratch, float* const* d_phase,
                            double* d_var, uint32_t* d_status, void* stream) {
  int rc = check_batch(plans, n);
  if (rc != EER4D_OK) return rc;
  if (!d_G || !d_aberr || !d_scratch) return EER4D_EINVAL;
  const float2* G[EER4D_MAX_SETS];
  for (int i = 0; i < n; ++i) {
    if (!d_G[i]) return EER4D_EINVAL;
    G[i] = static_cast<const float2*>(d_G[i]);
  }
  return cuda_fail(launch_trotter_batched(plans, G, n, d_aberr, d_scratch, d_phase, d_var,
                                          d_status, (cudaStream_t)stream));
}

int ssb_g_slices(const eer4d_plan* p, const void* d_G, const int32_t* h_bins, int n, void* d_out,
                 void* stream) {
  if (!p || !d_G || !h_bins || !d_out || n < 1 || n > EER4D_MAX_SLICES) return EER4D_EINVAL;
  for (int i = 0; i < n; ++i)
    if (h_bins[2 * i] < 0 || h_bins[2 * i] >= (int)p->g.scan_ny || h_bins[2 * i + 1] < 0 ||
        h_bins[2 * i + 1] >= (int)p->g.scan_nx)
      return EER4D_EINVAL;
  return cuda_fail(launch_g_slices(p, static_cast<const float2*>(d_G), h_bins, n,
                                   static_cast<float2*>(d_out), (cudaStream_t)stream));
}

// ---- launch-shape autotuner ------------------------------------------------
static bool tuning_ok(const eer4d_tuning* t) {
  const int tf = t->scatter_tf;
  if (tf != 0 && (tf < 4 || tf > 128 || (tf & (tf - 1)))) return false;
  return t->scatter_ctas_per_sm >= 0 && t->scatter_ctas_per_sm <= 32 && t->dft_ctas_per_sm >= 0 &&
         t->dft_ctas_per_sm <= 32 && t->trotter_ctas_per_sm >= 0 && t->trotter_ctas_per_sm <= 32;
}

int eer4d_set_tuning(eer4d_plan* p, const eer4d_tuning* t) {
  if (!p || !t || !tuning_ok(t)) return EER4D_EINVAL;
  p->tune = *t;
  return EER4D_OK;
}

int eer4d_get_tuning(const eer4d_plan* p, eer4d_tuning* t) {
  if (!p || !t) return EER4D_EINVAL;
  *t = p->tune;
  return EER4D_OK;
}

extern "C++" {
namespace {
// mean time of `reps` runs of fn after one untimed run; negative on a failure
template <typename Fn>
float time_ms(cudaStream_t s, int reps, Fn fn) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1.f; }
  float ms = -1.f;
  if (fn() == cudaSuccess && cudaEventRecord(a, s) == cudaSuccess) {
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r) ok = fn() == cudaSuccess;
    if (ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
        cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
      ms /= reps;
    else
      ms = -1.f;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}
}  // namespace
}  // extern "C++"

int eer4d_autotune(eer4d_plan* p, const uint32_t* d_idx, uint64_t n_idx, const uint64_t* d_off,
                   void* d_work, void* d_G, void* d_scratch, const double* d_aberr,
                   uint32_t* d_status, void* stream, eer4d_tuning* h_out) {
  if (!p || !d_off || (n_idx && !d_idx) || !d_work || !d_G || !d_scratch || !d_aberr)
    return EER4D_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // the caller's stage events stay out of the timing runs
  cudaEvent_t save_a[EER4D_N_STAGES], save_b[EER4D_N_STAGES];
  for (int i = 0; i < EER4D_N_STAGES; ++i) {
    save_a[i] = p->ev_start[i];
    save_b[i] = p->ev_stop[i];
    p->ev_start[i] = p->ev_stop[i] = nullptr;
  }
  __half* counts = static_cast<__half*>(d_work);
  float2* X1 = reinterpret_cast<float2*>(static_cast<unsigned char*>(d_work) +
                                         al256(work_counts_bytes(p)));
  float2* G = static_cast<float2*>(d_G);
  const eer4d_tuning keep = p->tune;
  eer4d_tuning best = keep;
  int rc = EER4D_OK;
  // scatter: frames per tile 16..128 (pixels chunked to fit) x 1..3 CTAs per SM
  {
    float tbest = -1.f;
    for (int tf = 16; tf <= 128; tf *= 2) {
      for (int cps = 1; cps <= 3; ++cps) {
        p->tune = best;
        p->tune.scatter_tf = tf;
        p->tune.scatter_ctas_per_sm = cps;
        const float ms = time_ms(s, 2, [&] {
          return launch_scatter(p, d_idx, n_idx, d_off, 0, (uint64_t)p->F, counts, d_status, s);
        });
        if (ms > 0.f && (tbest < 0.f || ms < tbest)) {
          tbest = ms;
          best.scatter_tf = tf;
          best.scatter_ctas_per_sm = cps;
        }
      }
    }
    best.ms[0] = tbest;
    p->tune = best;
    // counts of the chosen shape for the DFT runs below
    rc = cuda_fail(launch_scatter(p, d_idx, n_idx, d_off, 0, (uint64_t)p->F, counts, d_status, s));
  }
  // fused scan DFT: 1..4 CTAs per SM
  if (rc == EER4D_OK && dft2_fused_ok(p)) {
    unsigned* ctl = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(X1) +
                                                al256(dft2_ring_bytes(p)));
    float tbest = -1.f;
    for (int cps = 1; cps <= 4; ++cps) {
      p->tune = best;
      p->tune.dft_ctas_per_sm = cps;
      const float ms = time_ms(s, 2, [&] { return launch_dft2_fused(p, counts, X1, G, ctl, d_status, s); });
      if (ms > 0.f && (tbest < 0.f || ms < tbest)) {
        tbest = ms;
        best.dft_ctas_per_sm = cps;
      }
    }
    best.ms[1] = tbest;
    p->tune = best;
    rc = cuda_fail(launch_dft2_fused(p, counts, X1, G, ctl, d_status, s));
  } else if (rc == EER4D_OK) {
    rc = cuda_fail(launch_stage1(p, counts, X1, 0, (int)p->g.scan_ny, s));
    if (rc == EER4D_OK) rc = cuda_fail(launch_stage2(p, X1, G, s));
  }
  // trotter: 1..3 CTAs per SM, one candidate
  if (rc == EER4D_OK) {
    float tbest = -1.f;
    for (int cps = 1; cps <= 3; ++cps) {
      p->tune = best;
      p->tune.trotter_ctas_per_sm = cps;
      const float ms = time_ms(s, 2, [&] {
        return launch_trotter(p, G, d_aberr, 1, TROT_FWD, d_scratch, nullptr, nullptr, nullptr,
                              nullptr, nullptr, d_status, s);
      });
      if (ms > 0.f && (tbest < 0.f || ms < tbest)) {
        tbest = ms;
        best.trotter_ctas_per_sm = cps;
      }
    }
    best.ms[2] = tbest;
  }
  p->tune = rc == EER4D_OK ? best : keep;
  for (int i = 0; i < EER4D_N_STAGES; ++i) {
    p->ev_start[i] = save_a[i];
    p->ev_stop[i] = save_b[i];
  }
  if (rc == EER4D_OK) rc = cuda_fail(cudaStreamSynchronize(s));
  if (h_out) *h_out = p->tune;
  return rc;
}

int eer4d_selftest_wait(void* d_scratch, uint32_t* d_status, void* stream) {
  if (!d_scratch || !d_status) return EER4D_EINVAL;
  return cuda_fail(launch_wait_selftest(static_cast<unsigned*>(d_scratch), d_status,
                                        (cudaStream_t)stream));
}

int ssb_trotter_counts(const eer4d_plan* p, const double* d_aberr, int32_t* d_count,
                       void* d_scratch, void* stream) {
  if (!p || !d_aberr || !d_count || !d_scratch) return EER4D_EINVAL;
  return cuda_fail(launch_trotter(p, nullptr, d_aberr, 1, TROT_COUNT, d_scratch, nullptr, nullptr,
                                  nullptr, nullptr, d_count, nullptr, (cudaStream_t)stream));
}

}  // extern "C"
