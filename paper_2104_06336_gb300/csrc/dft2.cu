// Fused two-axis scan DFT of the G function (Sec. IV: G(k, K) is the Fourier
// transform of every detector pixel's image over the scan) for square
// power-of-two scans, N = scan_ny = scan_nx in {128, 256, 512, 1024}.
//
// The separable transform runs as one persistent launch over a queue of
// tiles.  Pixels are taken in groups of gp (8 or 16); for group g:
//   S1 tasks (one per scan row y): real-to-complex DFT along x of the gp
//      pixel rows at y, into ring slot g % 4, complex64 [nkx][N][gp];
//   S2 tasks (one per K_x): DFT along y of the slot's gp columns at K_x,
//      written transposed into G [nkx][P_pad][N]; the slot's lines are then
//      dropped from L2 without write-back (discard.global.L2).
// A slot is 8 pixels x N x (N/2 + 1) x 8 bytes (34 MB at N = 1024), so the
// two slots in use (one being written, one being read) stay in the 126 MB
// L2: the DRAM traffic is the fp16 counts read once and G written once,
// without the round trip of a full-size intermediate.  The ring has four
// slots so that S1(g) seldom waits for the slot's previous group (three slots
// measured 0.01 ms slower at N = 1024, two slots 0.5 ms slower).  Completion counts are published in batches (one
// fence and atomic per CTA and change of group), the queue is read two tasks
// ahead, and a CTA skips waits for groups it has already seen complete.  Tasks are handed out in the order S1(0), then
// S1(g+1), S2(g) for g = 0, 1, ...; S2(g) waits until all S1(g) tasks are
// done, S1(g) (g >= 4) until all S2(g-4) tasks are done (slot reuse).  Every
// task waits only on tasks handed out before it, so the queue needs no
// co-residency of CTAs.  Waits are bounded (1 s on %globaltimer and an
// iteration cap); a wait that gives up sets EER4D_ST_TIMEOUT and an abort
// flag that ends every CTA's loop.
#include <algorithm>

#include "fft_reg.cuh"

namespace {

#ifndef EER4D_DFT2_S1_WARP
#define EER4D_DFT2_S1_WARP 1  // N = 1024: warp-private four-step passes of the S1 tile
#endif

#ifndef EER4D_DFT2_MINB
#define EER4D_DFT2_MINB 4  // resident CTAs per SM the register budget is sized for
#endif

constexpr int kRing = 4;
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr unsigned kWaitIters = 1u << 24;

struct Dft2Params {
  int N, nkx, P_pad, gp, n_groups, n1, n2;
  long long slot;   // float2 per ring slot
  unsigned total;   // tasks (< 2^31)
  long long F;      // row stride of the counts (frames, padded)
};

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 only: waits until *cnt >= target.  False when the abort flag is set
// or the wait gives up (then it sets EER4D_ST_TIMEOUT and the abort flag).
__device__ bool wait_count(const unsigned* cnt, unsigned target, unsigned* abort_flag,
                           uint32_t* st) {
  if (ld_acquire(cnt) >= target) return true;
  const unsigned long long t0 = now_ns();
  for (unsigned it = 0; it < kWaitIters; ++it) {
    __nanosleep(128);
    if (ld_acquire(cnt) >= target) return true;
    if (ld_acquire(abort_flag)) return false;
    if (now_ns() - t0 > kWaitNs) break;
  }
  st_or(st, EER4D_ST_TIMEOUT);
  atomicExch(abort_flag, 1u);
  return false;
}

struct Task {
  int type;  // 0 = S1 (DFT along x of one scan row), 1 = S2 (DFT along y), -1 = queue empty
  int g;     // pixel group
  int r;     // index within the group's tasks of that type
};

// Queue index -> task (thread 0 only; 32-bit: the host keeps total < 2^31).
__device__ __forceinline__ Task decode(unsigned t, const Dft2Params& q) {
  if (t >= q.total) return Task{-1, 0, 0};
  const unsigned n1 = q.n1;
  if (t < n1) return Task{0, 0, (int)t};
  const unsigned u = t - n1;
  const unsigned pair = n1 + (unsigned)q.n2;
  const unsigned full = (unsigned)(q.n_groups - 1) * pair;
  if (u < full) {
    const unsigned g = u / pair;
    const unsigned r = u - g * pair;
    return r < n1 ? Task{0, (int)g + 1, (int)r} : Task{1, (int)g, (int)(r - n1)};
  }
  return Task{1, q.n_groups - 1, (int)(u - full)};
}

// Drops the L2 lines of [p, p + bytes) without writing them back (the slot
// is dead once its S2 task has read it); p and bytes are multiples of 128.
__device__ __forceinline__ void l2_discard(const void* p, size_t bytes, int tid, int nt) {
  const size_t base = __cvta_generic_to_global(p);
  for (size_t o = (size_t)tid * 128; o < bytes; o += (size_t)nt * 128)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(base + o) : "memory");
}

// Completion counts are published in batches: thread 0 holds the count of
// finished tasks of one (type, group) and publishes it (fence, then one
// atomic add) when its CTA moves to another (type, group), before any wait,
// and at exit, always after a CTA barrier that follows the tasks it counts.
struct Pending {
  int type, g;
  unsigned n;
};

__device__ __forceinline__ void publish(Pending& pd, unsigned* done1, unsigned* done2) {
  if (pd.n) {
    __threadfence();
    atomicAdd((pd.type == 0 ? done1 : done2) + pd.g, pd.n);
  }
  pd.n = 0;
  pd.type = pd.g = -1;
}

// S1 tile for N = 1024 (R1 = R2 = 32) with one warp per complex row pair:
// warp w transforms z = row(p0 + 2w) + i row(p0 + 2w + 1) of scan row r.
// Pass 1 (lane = j2) and pass 2 (lane = k1) exchange through the warp's own
// region of shared memory, so they need only __syncwarp; one CTA barrier then
// makes the CP spectra visible to the half-spectrum split, which writes the
// slot [k][r][GP] with one 16-byte store per (k, pair).
constexpr int kW32Pitch = 33;                 // pass-1 rows (k1) of 32 + 1 float2
constexpr int kW32Region = 32 * kW32Pitch + 4;  // float2 per warp (+4: pairs in distinct banks)

template <int CP>
__device__ __forceinline__ void s1_tile_w32(const __half* __restrict__ counts, float2* slot,
                                            const float2* __restrict__ tw4, int p0, int r,
                                            long long F, float2* sm) {
  constexpr int N = 1024, GP = 2 * CP, NT = 32 * CP;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* rg = sm + w * kW32Region;
  float2 v[32];
  {
    const __half* pa = counts + (size_t)(p0 + 2 * w) * F + (size_t)r * N + lane;
    const __half* pb = pa + F;
#pragma unroll
    for (int j1 = 0; j1 < 32; ++j1)
      v[j1] = make_float2(ld_h<true>(pa + 32 * j1), ld_h<true>(pb + 32 * j1));
  }
  dft_reg<32, 1>(v);
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1)
    rg[k1 * kW32Pitch + lane] = (k1 == 0) ? v[k1] : cmul(v[k1], __ldg(tw4 + k1 * 32 + lane));
  __syncwarp();
#pragma unroll
  for (int j2 = 0; j2 < 32; ++j2) v[j2] = rg[lane * kW32Pitch + j2];
  dft_reg<32, 1>(v);
  __syncwarp();  // every lane has read the region before it is overwritten
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) rg[lane + 32 * k2] = v[k2];  // Z(k1 + 32 k2)
  __syncthreads();
  constexpr int NK = N / 2 + 1;
  for (int i = threadIdx.x; i < NK * CP; i += NT) {
    const int b = i % CP, k = i / CP;
    const float2 z = sm[b * kW32Region + k];
    const float2 zm = sm[b * kW32Region + ((N - k) & (N - 1))];
    const float2 A = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    const float2 B = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    *reinterpret_cast<float4*>(slot + (size_t)k * N * GP + (size_t)r * GP + 2 * b) =
        make_float4(A.x, A.y, B.x, B.y);
  }
}

template <int R1, int R2, int CP>
__global__ void __launch_bounds__(R1 * CP, EER4D_DFT2_MINB * 128 / (R1 * CP))
    k_dft2_fused(const __half* __restrict__ counts, float2* ring, float2* G,
                 const float2* __restrict__ twx4, const float2* __restrict__ twy4, Dft2Params q,
                 unsigned* ctl, uint32_t* st) {
  constexpr int NT = R1 * CP;
  constexpr int N = R1 * R2;  // = q.N
  constexpr int GP = 2 * CP;  // pixels per group, = q.gp
  extern __shared__ float2 sm[];
  __shared__ Task s_k[3];
  __shared__ int s_ok;
  unsigned* next = ctl;
  unsigned* abort_flag = ctl + 1;
  unsigned* done1 = ctl + 2;
  unsigned* done2 = done1 + q.n_groups;
  // thread 0's bookkeeping lives in shared memory (no registers in the tiles)
  __shared__ Pending pd;
  __shared__ int known1, known2;  // groups seen complete (S1, S2)
  // The queue is read two tasks ahead: the index taken in iteration i is kept
  // in a register and decoded into s_k for iteration i + 2 only in iteration
  // i + 1, so thread 0 never waits for the atomic's reply.
  unsigned inflight = 0;
  if (threadIdx.x == 0) {
    pd.type = pd.g = -1;
    pd.n = 0;
    known1 = known2 = -1;
    s_k[0] = decode(atomicAdd(next, 1u), q);
    s_k[1] = decode(atomicAdd(next, 1u), q);
  }
  for (int it = 0;; ++it) {
    __syncthreads();  // the previous task is finished by every thread
    const Task k = s_k[it % 3];
    if (k.type < 0) break;
    if (threadIdx.x == 0) {
      // the publish fence first: it then waits only for the previous task's
      // writes, not for the queue atomic issued below
      if (pd.n && (pd.type != k.type || pd.g != k.g)) publish(pd, done1, done2);
      if (it > 0) s_k[(it + 1) % 3] = decode(inflight, q);
      inflight = atomicAdd(next, 1u);
      bool ok = true;
      if (k.type == 1 && k.g > known1) {
        publish(pd, done1, done2);
        ok = wait_count(done1 + k.g, (unsigned)q.n1, abort_flag, st);
        known1 = k.g;
      } else if (k.type == 0 && k.g >= kRing && k.g - kRing > known2) {
        publish(pd, done1, done2);
        ok = wait_count(done2 + (k.g - kRing), (unsigned)q.n2, abort_flag, st);
        known2 = k.g - kRing;
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    // debug build: the decoded task lies inside the group, row and K_x ranges (CTA-uniform)
    if (!EER4D_IN_RANGE(k.g, q.n_groups, st) || !EER4D_IN_RANGE(k.r, k.type ? q.n2 : q.n1, st))
      continue;
    {
      // the next task is known: if it is a DFT along x, pull its counts rows
      // (GP rows of 2N bytes) from DRAM into L2 now, so its loads hit L2
      const Task kn = s_k[(it + 1) % 3];
      if (kn.type == 0) {
        constexpr int lines = N / 64;  // 128-byte lines per row
        for (int i = threadIdx.x; i < GP * lines; i += NT) {
          const int row = i / lines, line = i - row * lines;
          const __half* a = counts + (size_t)(kn.g * GP + row) * q.F + (size_t)kn.r * N + line * 64;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
        }
      }
    }
    float2* slot = ring + (long long)(k.g % kRing) * q.slot;
    const int p0 = k.g * GP;
    if (k.type == 0) {
      // S1: the GP pixel rows of scan row r, DFT along x into the slot
      if constexpr (R1 == 32 && R2 == 32 && EER4D_DFT2_S1_WARP)
        s1_tile_w32<CP>(counts, slot, twx4, p0, k.r, q.F, sm);
      else
        rowfft_r2c_tile<R1, R2, CP, true, true>(counts, slot, twx4, q.P_pad, p0, p0, k.r, q.F, N,
                                                (long long)N * GP, 1, GP, sm);
    } else {
      // S2: all GP pixel columns of K_x = r, DFT along y into G, CP at a time
      const float2* blk = slot + (long long)k.r * N * GP;
      float2* gout = G + ((long long)k.r * q.P_pad + p0) * N;
#pragma unroll
      for (int c0 = 0; c0 < GP; c0 += CP) {
        if (c0) __syncthreads();
        colfft_tile<R1, R2, CP, 1, true, true>(blk, gout, twy4, c0, GP, GP, N, 1.f, sm);
      }
      // every load of the block happens in a first pass, before the tile's
      // barrier, so every thread is past the block's last read here
      l2_discard(blk, sizeof(float2) * (size_t)N * GP, threadIdx.x, NT);
    }
    if (threadIdx.x == 0) {
      pd.type = k.type;
      pd.g = k.g;
      ++pd.n;
    }
  }
  if (threadIdx.x == 0) publish(pd, done1, done2);  // after the loop's last barrier
}

template <int R1, int R2, int CP>
cudaError_t launch_t(const eer4d_plan* p, const __half* counts, float2* ring, float2* G,
                     unsigned* ctl, size_t ctl_bytes, uint32_t* st, cudaStream_t s) {
  constexpr int N = R1 * R2, NT = R1 * CP;
  const size_t a = (size_t)R1 * CP * (R2 + 1) + 2 * CP, b = (size_t)N * CP;
  const size_t c = (size_t)CP * kW32Region;
  const size_t sm = sizeof(float2) * std::max(std::max(a, b), c);
  auto kern = k_dft2_fused<R1, R2, CP>;
  cudaError_t e = ensure_smem((const void*)kern, sm);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, sm)) != cudaSuccess)
    return e;
  Dft2Params q;
  q.N = N;
  q.nkx = p->nkx;
  q.P_pad = p->P_pad;
  q.gp = 2 * CP;
  q.n_groups = p->P_pad / q.gp;
  q.n1 = N;
  q.n2 = p->nkx;
  q.slot = (long long)p->nkx * N * q.gp;
  const long long total = (long long)q.n_groups * (q.n1 + q.n2);
  if (total >= (1ll << 31)) return cudaErrorInvalidValue;
  q.total = (unsigned)total;
  q.F = p->cstride;
  if ((e = cudaMemsetAsync(ctl, 0, ctl_bytes, s)) != cudaSuccess) return e;
  int cps = per_sm > 0 ? per_sm : 1;
  if (p->tune.dft_ctas_per_sm > 0 && p->tune.dft_ctas_per_sm < cps) cps = p->tune.dft_ctas_per_sm;
  long long grid = (long long)cps * nsm;
  if (grid > (long long)q.total) grid = q.total;
  if (!p->fx.tw4 || !p->fy.tw4) return cudaErrorInvalidValue;
  k_dft2_fused<R1, R2, CP><<<(unsigned)grid, NT, sm, s>>>(counts, ring, G, p->fx.tw4, p->fy.tw4, q,
                                                          ctl, st);
  count_launches(1);
  return cudaGetLastError();
}

// The wait above on a counter that nothing increments: it must give up after
// its time limit and report EER4D_ST_TIMEOUT (tests of the failure path).
__global__ void k_wait_selftest(unsigned* ctl, uint32_t* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) wait_count(ctl, 1u, ctl + 1, st);
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned* ctl, uint32_t* st, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  k_wait_selftest<<<1, 32, 0, s>>>(ctl, st);
  count_launches(1);
  return cudaGetLastError();
}

bool dft2_fused_ok(const eer4d_plan* p) {
  const int N = (int)p->g.scan_nx;
  return p->precision == EER4D_FP32_FFT && p->g.scan_ny == p->g.scan_nx &&
         (N == 128 || N == 256 || N == 512 || N == 1024);
}

#ifndef EER4D_DFT2_CP_LARGE
#define EER4D_DFT2_CP_LARGE 4  // pixel pairs per S1 tile (= columns per S2 call) for N >= 512
#endif
static int dft2_gp(int N) { return N >= 512 ? 2 * EER4D_DFT2_CP_LARGE : 16; }

size_t dft2_ring_bytes(const eer4d_plan* p) {
  const int N = (int)p->g.scan_nx;
  return sizeof(float2) * (size_t)kRing * p->nkx * N * dft2_gp(N);
}

size_t dft2_ctl_bytes(const eer4d_plan* p) {
  const int n_groups = p->P_pad / dft2_gp((int)p->g.scan_nx);
  return sizeof(unsigned) * (size_t)(2 + 2 * n_groups);
}

cudaError_t launch_dft2_fused(const eer4d_plan* p, const __half* counts, float2* ring, float2* G,
                              unsigned* ctl, uint32_t* st, cudaStream_t s) {
  const size_t cb = dft2_ctl_bytes(p);
  stage_begin(p, EER4D_STAGE_DFT_XY, s);
  cudaError_t e;
  switch (p->g.scan_nx) {
    case 1024: e = launch_t<32, 32, EER4D_DFT2_CP_LARGE>(p, counts, ring, G, ctl, cb, st, s); break;
    case 512: e = launch_t<32, 16, EER4D_DFT2_CP_LARGE>(p, counts, ring, G, ctl, cb, st, s); break;
    case 256: e = launch_t<16, 16, 8>(p, counts, ring, G, ctl, cb, st, s); break;
    default: e = launch_t<16, 8, 8>(p, counts, ring, G, ctl, cb, st, s); break;
  }
  stage_end(p, EER4D_STAGE_DFT_XY, s);
  return e;
}
