// Transform kernels of the pipeline (everything except the per-bin
// contractions): twiddle table, batched zero-padded real FFT (Alg. 2, steps
// 1-2), the stage-1 -> stage-2 retransform (Alg. 2 steps 4-5 for F_G, the
// D_t stencil of Sec. II-B.2, then steps 1-2 for F_q), the split-K reduction
// of stage-2 partials fused with the final IFFT + Truncate, and the load-time
// conversion of FP32 spectra into the resident storage types.
#include "fft.cuh"

namespace s2w {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;

// tw[m] = exp(-2 pi i m / L), m < L, evaluated in FP64 and stored as FP32.
__global__ void k_twiddles(float2* tw, int L) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  double s, c;
  sincospi(2.0 * static_cast<double>(m) / static_cast<double>(L), &s, &c);
  tw[m] = make_float2(static_cast<float>(c), static_cast<float>(-s));
}

template <int P>
__device__ __forceinline__ void load_twiddles(float2* tw, const float2* __restrict__ twg) {
  for (int m = threadIdx.x; m < 64 * P; m += blockDim.x) tw[m] = twg[m];
}

// One warp per row: x[row][0..n_in) zero-padded to L = 2N, bins 0..N to
// X[l * ld_l + (row / rows_a) * ld_a + row % rows_a].
template <int P>
__global__ void __launch_bounds__(kThreads) k_rfft_rows(const float* __restrict__ x, long long rows, int n_in,
                                                        const float2* __restrict__ twg, float2* __restrict__ X,
                                                        long long ld_l, long long rows_a, long long ld_a,
                                                        const int* __restrict__ lens) {
  constexpr int N = 32 * P;
  constexpr int L = 2 * N;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* tw = reinterpret_cast<float2*>(smraw);
  float2* zs = tw + L + (threadIdx.x >> 5) * N;
  load_twiddles<P>(tw, twg);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long row = static_cast<long long>(blockIdx.x) * kWarps + (threadIdx.x >> 5);
  if (row >= rows) return;
  const float* xr = x + row * n_in;
  // lens: active samples per group of rows_a rows (later samples read as 0)
  const int n_act = lens != nullptr ? min(n_in, max(0, __ldg(lens + row / rows_a))) : n_in;
  const FftLane<P> fl = fft_lane<P>(tw, lane);
  warp_rfft_stage<P>([&](int n) { return n < n_act ? __ldg(xr + n) : 0.f; }, zs, tw, fl, lane);
  float2* out = X + (row / rows_a) * ld_a + (row % rows_a);
  for (int k = lane; k <= N; k += 32) out[k * ld_l] = rfft_bin<P>(zs, tw, k);
}

// One warp per row: bins X[row][0..N] -> first N samples x[row][0..N).
template <int P>
__global__ void __launch_bounds__(kThreads) k_irfft_rows(const float2* __restrict__ X, long long rows,
                                                         const float2* __restrict__ twg, float* __restrict__ x) {
  constexpr int N = 32 * P;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* tw = reinterpret_cast<float2*>(smraw);
  float2* scr = tw + 2 * N + (threadIdx.x >> 5) * N;
  load_twiddles<P>(tw, twg);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long row = static_cast<long long>(blockIdx.x) * kWarps + (threadIdx.x >> 5);
  if (row >= rows) return;
  const float2* xr = X + row * (N + 1);
  float* out = x + row * N;
  const FftLane<P> fl = fft_lane<P>(tw, lane);
  warp_irfft_head<P>([&](int k) { return xr[k]; }, [&](int n, float v) { out[n] = v; }, tw, fl, lane, scr);
}

// Retransform of 32 consecutive grid points per CTA, rupture blockIdx.y:
//   mhat[l][i] (bins 0..N)  -> IFFT, keep n < N (Truncate)  -> m
//   v = D_t m  (backward difference; or v = m when dt_mode is NONE)
//   v zero-padded to 2N -> FFT -> vhat[l][i]  (FP32, or BF16 pairs when BF16OUT).
// Optionally writes m to seafloor[i][0..N).
template <int P, bool BF16OUT>
__global__ void __launch_bounds__(kThreads) k_retransform(const float2* __restrict__ mhat, long long Ng, long long ld_m,
                                                          const float2* __restrict__ twg, float inv_dt, int dt_mode,
                                                          void* __restrict__ vout, long long ld_v,
                                                          float* __restrict__ seafloor, long long mhat_ld_b,
                                                          long long vhat_ld_b, __nv_bfloat162* __restrict__ vout_lo,
                                                          int n_alloc) {
  constexpr int N = 32 * P;
  constexpr int L = 2 * N;
  constexpr int NB = N + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* tw = reinterpret_cast<float2*>(smraw);
  float2* tile = tw + L;                                 // [32][NB]
  float2* zs = tile + 32 * NB + (threadIdx.x >> 5) * N;  // per warp [N]
  float* mb = reinterpret_cast<float*>(tile + 32 * NB + kWarps * N) + (threadIdx.x >> 5) * N;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const long long i0 = static_cast<long long>(blockIdx.x) * 32;
  mhat += blockIdx.y * mhat_ld_b;
  if (seafloor != nullptr) seafloor += static_cast<long long>(blockIdx.y) * Ng * N;
  load_twiddles<P>(tw, twg);
  // 16 independent loads in flight per thread (a warp reads 256 contiguous
  // bytes of one bin per load)
  constexpr int kU = 16;
  for (int e0 = threadIdx.x; e0 < NB * 32; e0 += kThreads * kU) {
    float2 v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * kThreads;
      const int l = e >> 5, c = e & 31;
      const long long i = i0 + c;
      v[u] = (e < NB * 32 && i < Ng) ? __ldg(mhat + l * ld_m + i) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * kThreads;
      if (e < NB * 32) tile[(e & 31) * NB + (e >> 5)] = v[u];
    }
  }
  __syncthreads();
  const FftLane<P> fl = fft_lane<P>(tw, lane);
  for (int c = warp; c < 32; c += kWarps) {
    const long long i = i0 + c;
    if (i >= Ng) break;
    float2* X = tile + c * NB;
    // m[n] lives at mb[msw(n)]: the IFFT hands the lanes samples 2 fft_out
    // (+1) in a strided pattern; the XOR swizzle inside blocks of 32 floats
    // spreads those stores (and the later natural-order reads) over the banks
    auto msw = [](int n) { return n ^ (((n >> 5) ^ (n >> 7)) & 31); };
    warp_irfft_head<P>([&](int k) { return X[k]; }, [&](int n, float v) { mb[msw(n)] = v; }, tw, fl, lane, zs);
    __syncwarp();
    if (seafloor != nullptr)
      for (int n = lane; n < N; n += 32) seafloor[i * N + n] = mb[msw(n)];
    if (dt_mode == S2W_DT_NONE) {
      warp_rfft_stage<P>([&](int n) { return n < N ? mb[msw(n)] : 0.f; }, zs, tw, fl, lane);
    } else if (dt_mode == kDtTranspose) {
      // D_t^T: u[n] = (w[n] - w[n+1]) / dt, w[N] = 0
      warp_rfft_stage<P>(
          [&](int n) { return n < N ? (mb[msw(n)] - (n + 1 < N ? mb[msw(n + 1)] : 0.f)) * inv_dt : 0.f; }, zs, tw,
          fl, lane);
    } else {
      warp_rfft_stage<P>(
          [&](int n) { return n < N ? (mb[msw(n)] - (n > 0 ? mb[msw(n - 1)] : 0.f)) * inv_dt : 0.f; }, zs, tw, fl,
          lane);
    }
    for (int k = lane; k <= N; k += 32) X[k] = rfft_bin<P>(zs, tw, k);
    __syncwarp();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NB * 32; e += kThreads) {
    const int l = e >> 5, c = e & 31;
    const long long i = i0 + c;
    if (i >= Ng) continue;
    const float2 v = tile[c * NB + l];
    if (BF16OUT && n_alloc > 0) {
      // B operand of the conjugate embedding (tensor-engine adjoint): rows
      // 2b = (Re v, Im v) and 2b+1 = (Im v, -Re v) of [l][n_alloc][ld_v]
      const long long o0 = (static_cast<long long>(l) * n_alloc + 2 * blockIdx.y) * ld_v + i;
      const float2 r[2] = {make_float2(v.x, v.y), make_float2(v.y, -v.x)};
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(r[h2].x, r[h2].y);
        static_cast<__nv_bfloat162*>(vout)[o0 + h2 * ld_v] = h;
        if (vout_lo != nullptr)
          vout_lo[o0 + h2 * ld_v] = __floats2bfloat162_rn(r[h2].x - __low2float(h), r[h2].y - __high2float(h));
      }
    } else if (BF16OUT) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
      (static_cast<__nv_bfloat162*>(vout) + blockIdx.y * vhat_ld_b)[l * ld_v + i] = h;
      if (vout_lo != nullptr)  // low-order part: v - hi, rounded again
        (vout_lo + blockIdx.y * vhat_ld_b)[l * ld_v + i] =
            __floats2bfloat162_rn(v.x - __low2float(h), v.y - __high2float(h));
    } else
      (static_cast<float2*>(vout) + blockIdx.y * vhat_ld_b)[l * ld_v + i] = v;
  }
}

// Split-K reduction + output transform, one CTA per (rupture b, observation o):
//   Qhat[l] = sum_{s < nseg} part[b*s_b + l*s_l + s*s_s + o]   (fixed order:
// deterministic), all bins in parallel over the CTA's threads, then one warp
// forms q[b][o][n] = IFFT(Qhat)[n], n < N.
template <int P>
__global__ void __launch_bounds__(kThreads) k_reduce_irfft(const float2* __restrict__ part, int No, int nseg,
                                                           long long s_b, long long s_l, long long s_s,
                                                           const float2* __restrict__ twg, float* __restrict__ q,
                                                           int n_keep) {
  constexpr int N = 32 * P;
  constexpr int L = 2 * N;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* tw = reinterpret_cast<float2*>(smraw);
  float2* xs = tw + L;
  float2* scr = xs + N + 1;
  load_twiddles<P>(tw, twg);
  const int b = blockIdx.x / No, o = blockIdx.x % No;
  const float2* pb = part + b * s_b + o;
  for (int k = threadIdx.x; k <= N; k += kThreads) {
    const float2* pk = pb + static_cast<long long>(k) * s_l;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int s = 0; s < nseg; ++s) acc = cadd(acc, pk[static_cast<long long>(s) * s_s]);
    xs[k] = acc;
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  float* out = q + static_cast<long long>(blockIdx.x) * n_keep;
  const FftLane<P> fl = fft_lane<P>(tw, threadIdx.x);
  warp_irfft_head<P>([&](int k) { return xs[k]; },
                     [&](int n, float v) {
                       if (n < n_keep) out[n] = v;
                     },
                     tw, fl, threadIdx.x, scr);
}

// part[l][s][e] (l < Nb, s < nseg, e < per): part[l][0][e] becomes the sum
// over s in increasing order (the order k_reduce_irfft adds them in), read
// coalesced along e, so that the reduction reads one segment.
__global__ void k_sum_chunks(float2* __restrict__ part, int Nb, int nseg, long long per) {
  const long long total = static_cast<long long>(Nb) * per;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    float2* p = part + (e / per) * nseg * per + e % per;
    float2 acc = make_float2(0.f, 0.f);
    for (int s = 0; s < nseg; ++s) acc = cadd(acc, p[static_cast<long long>(s) * per]);
    p[0] = acc;
  }
}

// X[l][r] *= (1 - W_L^l) / dt for l <= L/2, r < per_bin: the spectrum of the
// backward difference, folded into the stage-2 spectra of the single-pass
// variant (no retransform between the stages; L = 4 Nt leaves no wrap).
__global__ void k_scale_dt(float2* __restrict__ X, int Nb, long long per_bin, const float2* __restrict__ twg,
                           float inv_dt) {
  const long long total = static_cast<long long>(Nb) * per_bin;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int l = static_cast<int>(e / per_bin);
    const float2 w = twg[l];
    const float2 d = make_float2((1.f - w.x) * inv_dt, -w.y * inv_dt);
    X[e] = cmul(X[e], d);
  }
}

// FP32 spectra -> resident storage (FP32 / BF16 / BF16 hi+lo), block copy:
// dst[l * ld_dst_l + dst_off + r] = convert(src[l * n_per_l + r]).
__global__ void k_store_blocks(const float2* __restrict__ src, int Nb, long long n_per_l, int el, void* dst,
                               void* dst_lo, long long ld_dst_l, long long dst_off) {
  const long long total = static_cast<long long>(Nb) * n_per_l;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long l = e / n_per_l, r = e % n_per_l;
    const float2 v = src[e];
    const long long d = l * ld_dst_l + dst_off + r;
    if (el == EL_FP32) {
      static_cast<float2*>(dst)[d] = v;
    } else {
      const __nv_bfloat162 hi = __floats2bfloat162_rn(v.x, v.y);
      static_cast<__nv_bfloat162*>(dst)[d] = hi;
      if (el == EL_BF16_HILO) {
        const float2 h = __bfloat1622float2(hi);
        static_cast<__nv_bfloat162*>(dst_lo)[d] = __floats2bfloat162_rn(v.x - h.x, v.y - h.y);
      }
    }
  }
}

// Stage-2 spectra, staging [l][o][nc] -> resident [l][seg][o][RL] at grid
// column i = c0 + c (seg = i / RL).
__global__ void k_store_adjoint(const float2* __restrict__ src, int Nb, int No, long long nc, long long c0, int RL,
                                int nseg, int el, void* dst) {
  const long long total = static_cast<long long>(Nb) * No * nc;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long l = e / (No * nc);
    const long long rem = e % (No * nc);
    const long long o = rem / nc, c = rem % nc;
    const long long i = c0 + c;
    const long long d = ((l * nseg + i / RL) * No + o) * RL + (i % RL);
    const float2 v = src[e];
    if (el == EL_FP32)
      static_cast<float2*>(dst)[d] = v;
    else
      static_cast<__nv_bfloat162*>(dst)[d] = __floats2bfloat162_rn(v.x, v.y);
  }
}

// FP8 scales: one CTA per (bin l, 256-row block) of the staging chunk
// [l][rows][Ns_pad]; amax over |Re|, |Im| of the block, then, in FP64,
// scale = amax / 448 (448 = largest finite e4m3).
__global__ void k_fp8_scales(const float2* __restrict__ spec, long long rows, int Ns_pad, long long row0, float* scale,
                             int nblk) {
  const int l = blockIdx.y;
  const long long rb = static_cast<long long>(blockIdx.x) * 256;
  const long long re = min(rows, rb + 256);
  const float2* base = spec + (static_cast<long long>(l) * rows + rb) * Ns_pad;
  const long long n = (re - rb) * Ns_pad;
  float m = 0.f;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    const float2 v = base[e];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = 0.f;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) mm = fmaxf(mm, red[w]);
    const double s = static_cast<double>(mm) / 448.0;
    scale[static_cast<long long>(l) * nblk + (row0 + rb) / 256] = static_cast<float>(s);
  }
}

// FP8 quantisation with round-to-nearest-even and saturation:
// dst[l][row0 + r][j] = e4m3(spec[l][r][j] / scale[l][(row0 + r) / 256]).
__global__ void k_fp8_quantize(const float2* __restrict__ spec, int Nb, long long rows, int Ns_pad, long long row0,
                               long long Ng, const float* __restrict__ scale, int nblk,
                               __nv_fp8x2_storage_t* __restrict__ dst) {
  const long long per_l = rows * Ns_pad;
  const long long total = static_cast<long long>(Nb) * per_l;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long l = e / per_l, rem = e % per_l;
    const long long r = rem / Ns_pad;
    const float sc = scale[l * nblk + (row0 + r) / 256];
    const float inv = sc > 0.f ? static_cast<float>(1.0 / static_cast<double>(sc)) : 0.f;
    const float2 v = spec[e];
    dst[l * Ng * Ns_pad + row0 * Ns_pad + rem] =
        __nv_cvt_float2_to_fp8x2(make_float2(v.x * inv, v.y * inv), __NV_SATFINITE, __NV_E4M3);
  }
}

// Residual and misfit: r = q - d in place of q, loss[b] = 0.5 sum r^2 over the
// rupture's No x Nt samples (one CTA per rupture, fixed summation order).
__global__ void __launch_bounds__(kThreads) k_residual(float* __restrict__ q, const float* __restrict__ d,
                                                       long long n_per_b, float* __restrict__ loss) {
  const long long base = static_cast<long long>(blockIdx.x) * n_per_b;
  float acc = 0.f;
  for (long long e = threadIdx.x; e < n_per_b; e += kThreads) {
    const float r = q[base + e] - d[base + e];
    q[base + e] = r;
    acc = fmaf(r, r, acc);
  }
  __shared__ float red[kWarps];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && loss != nullptr) {
    float t = 0.f;
    for (int w = 0; w < kWarps; ++w) t += red[w];
    loss[blockIdx.x] = 0.5f * t;
  }
}

int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g > 152LL * 32) g = 152LL * 32;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

template <int P>
size_t smem_retransform() {
  constexpr int N = 32 * P;
  return sizeof(float2) * (2 * N + 32 * (N + 1) + kWarps * N) + sizeof(float) * kWarps * N;
}

}  // namespace

#define S2W_DISPATCH_P(Nt, ...)                               \
  switch (Nt) {                                               \
    case 32: { constexpr int P = 1; __VA_ARGS__; } break;     \
    case 64: { constexpr int P = 2; __VA_ARGS__; } break;     \
    case 128: { constexpr int P = 4; __VA_ARGS__; } break;    \
    case 256: { constexpr int P = 8; __VA_ARGS__; } break;    \
    case 512: { constexpr int P = 16; __VA_ARGS__; } break;   \
    default: return cudaErrorInvalidValue;                    \
  }

cudaError_t launch_residual(float* q, const float* d, int B, long long n_per_b, float* loss, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_residual<<<B, kThreads, 0, st>>>(q, d, n_per_b, loss);
  return cudaGetLastError();
}

cudaError_t launch_twiddles(float2* tw, int L, cudaStream_t st) {
  k_twiddles<<<(L + 255) / 256, 256, 0, st>>>(tw, L);
  return cudaGetLastError();
}

cudaError_t launch_rfft_rows(const float* x, long long rows, int n_in, int Nt, const float2* tw, float2* X,
                             long long ld_l, long long rows_a, long long ld_a, cudaStream_t st, const int* lens) {
  if (rows <= 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((rows + kWarps - 1) / kWarps);
  S2W_DISPATCH_P(Nt, {
    const size_t sm = sizeof(float2) * (64 * P + kWarps * 32 * P);
    k_rfft_rows<P><<<grid, kThreads, sm, st>>>(x, rows, n_in, tw, X, ld_l, rows_a, ld_a, lens);
  });
  return cudaGetLastError();
}

cudaError_t launch_irfft_rows(const float2* X, long long rows, int Nt, const float2* tw, float* x, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((rows + kWarps - 1) / kWarps);
  S2W_DISPATCH_P(Nt, {
    const size_t sm = sizeof(float2) * (64 * P + kWarps * 32 * P);
    k_irfft_rows<P><<<grid, kThreads, sm, st>>>(X, rows, tw, x);
  });
  return cudaGetLastError();
}

cudaError_t launch_retransform(const float2* mhat, long long Ng, long long ld_m, int Nt, const float2* tw,
                               float inv_dt, int dt_mode, float2* vhat, long long ld_v, float* seafloor,
                               cudaStream_t st, int nb, long long mhat_ld_b, long long vhat_ld_b,
                               __nv_bfloat162* vhat_bf, __nv_bfloat162* vhat_bf_lo, int n_alloc) {
  if (Ng <= 0 || nb <= 0) return cudaSuccess;
  const dim3 grid(static_cast<unsigned>((Ng + 31) / 32), static_cast<unsigned>(nb));
  S2W_DISPATCH_P(Nt, {
    const size_t sm = smem_retransform<P>();
    if (vhat_bf != nullptr) {
      cudaError_t e = cudaFuncSetAttribute(k_retransform<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(sm));
      if (e != cudaSuccess) return e;
      k_retransform<P, true><<<grid, kThreads, sm, st>>>(mhat, Ng, ld_m, tw, inv_dt, dt_mode, vhat_bf, ld_v, seafloor,
                                                         mhat_ld_b, vhat_ld_b, vhat_bf_lo, n_alloc);
    } else {
      cudaError_t e = cudaFuncSetAttribute(k_retransform<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(sm));
      if (e != cudaSuccess) return e;
      k_retransform<P, false><<<grid, kThreads, sm, st>>>(mhat, Ng, ld_m, tw, inv_dt, dt_mode, vhat, ld_v, seafloor,
                                                          mhat_ld_b, vhat_ld_b, nullptr, 0);
    }
  });
  return cudaGetLastError();
}

cudaError_t launch_reduce_irfft(const float2* part, int B, int No, int nseg, int Nt, long long s_b, long long s_l,
                                long long s_s, const float2* tw, float* q, cudaStream_t st, int n_keep) {
  if (n_keep <= 0 || n_keep > Nt) n_keep = Nt;
  const long long n = static_cast<long long>(B) * No;
  if (n <= 0) return cudaSuccess;
  S2W_DISPATCH_P(Nt, {
    const size_t sm = sizeof(float2) * (64 * P + 32 * P + 1 + 32 * P);
    k_reduce_irfft<P><<<static_cast<unsigned>(n), kThreads, sm, st>>>(part, No, nseg, s_b, s_l, s_s, tw, q, n_keep);
  });
  return cudaGetLastError();
}

cudaError_t launch_sum_chunks(float2* part, int Nb, int nseg, long long per, cudaStream_t st) {
  k_sum_chunks<<<grid_for(Nb * per, 256), 256, 0, st>>>(part, Nb, nseg, per);
  return cudaGetLastError();
}

cudaError_t launch_scale_dt(float2* X, int Nb, long long per_bin, const float2* tw, float inv_dt, cudaStream_t st) {
  k_scale_dt<<<grid_for(Nb * per_bin, 256), 256, 0, st>>>(X, Nb, per_bin, tw, inv_dt);
  return cudaGetLastError();
}

cudaError_t launch_store_blocks(const float2* src, int Nb, long long n_per_l, int el, void* dst, void* dst_lo,
                                long long ld_dst_l, long long dst_off, cudaStream_t st) {
  k_store_blocks<<<grid_for(Nb * n_per_l, 256), 256, 0, st>>>(src, Nb, n_per_l, el, dst, dst_lo, ld_dst_l, dst_off);
  return cudaGetLastError();
}

cudaError_t launch_store_adjoint(const float2* src, int Nb, int No, long long nc, long long c0, int RL, int nseg,
                                 int el, void* dst, cudaStream_t st) {
  k_store_adjoint<<<grid_for(static_cast<long long>(Nb) * No * nc, 256), 256, 0, st>>>(src, Nb, No, nc, c0, RL, nseg,
                                                                                        el, dst);
  return cudaGetLastError();
}

cudaError_t launch_fp8_store(const float2* spec, int Nb, long long rows, int Ns_pad, long long row0, long long Ng,
                             float* scale, int nblk, void* dst, cudaStream_t st) {
  dim3 g(static_cast<unsigned>((rows + 255) / 256), static_cast<unsigned>(Nb));
  k_fp8_scales<<<g, 256, 0, st>>>(spec, rows, Ns_pad, row0, scale, nblk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fp8_quantize<<<grid_for(Nb * rows * Ns_pad, 256), 256, 0, st>>>(spec, Nb, rows, Ns_pad, row0, Ng, scale, nblk,
                                                                     static_cast<__nv_fp8x2_storage_t*>(dst));
  return cudaGetLastError();
}

}  // namespace s2w
