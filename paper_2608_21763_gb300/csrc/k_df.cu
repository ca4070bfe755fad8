// Transforms of the FP32_HILO (FP32 pair) storage precision: the same steps
// as k_fft.cu's kernels (Alg. 2 steps 1-2, the retransform between the
// stages with the D_t stencil of Sec. II-B.2, the split-K reduction with
// the final IFFT + Truncate), but with every spectrum and every sum carried
// as a double-float pair (df.cuh), so that the rounding of the transforms
// sits near 2^-48 of the signal instead of 2^-24.
//
// Why the pairs: an FFT evaluation rounds relative to the whole 2 Nt-sample
// window, spread evenly over all its samples; when most of a waveform's
// energy arrives after the kept Nt samples (a late arrival), the kept head
// is small against the window and its relative error grows by the ratio of
// the two.  Carrying every spectrum, sum and stored operator as hi + lo
// pairs takes that error down by 2^24.
//
// The transforms are plain DFT sums (one thread per output, twiddles from a
// double-float table), O(Nt^2) per signal: this precision serves accuracy,
// and its time goes to streaming the doubled operator spectra.
#include "df.cuh"
#include "s2w_internal.cuh"

namespace s2w {

namespace {

constexpr int kDfThreads = 256;

__device__ __forceinline__ dfl tw_re(const float4& w) { return {w.x, w.y}; }
__device__ __forceinline__ dfl tw_im(const float4& w) { return {w.z, w.w}; }

// tw[m] = exp(-2 pi i m / L) as (re hi, re lo, im hi, im lo), evaluated in
// FP64 and split into FP32 pairs.
__global__ void k_twiddles_df(float4* tw, int L) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  double s, c;
  sincospi(2.0 * static_cast<double>(m) / static_cast<double>(L), &s, &c);
  const double im = -s;
  const float ch = static_cast<float>(c), ih = static_cast<float>(im);
  tw[m] = make_float4(ch, static_cast<float>(c - static_cast<double>(ch)), ih,
                      static_cast<float>(im - static_cast<double>(ih)));
}

__device__ __forceinline__ void load_tw(float4* tws, const float4* __restrict__ tw, int L) {
  for (int m = threadIdx.x; m < L; m += blockDim.x) tws[m] = tw[m];
}

// X_l = sum_{n < n_act} x[n] exp(-2 pi i n l / L), l = 0..L/2, of FP32 rows
// x[row][0..n_in) (later samples, and those past lens[row / rows_a], read as
// zero).  Bin l of row `row` goes to X / X_lo[l * ld_l + (row / rows_a) *
// ld_a + row % rows_a] (hi and lo parts of re and im).  CTAs loop over rows.
__global__ void __launch_bounds__(kDfThreads) k_df_rfft_rows(const float* __restrict__ x, long long rows, int n_in,
                                                             int L, const float4* __restrict__ tw, float2* X,
                                                             float2* X_lo, long long ld_l, long long rows_a,
                                                             long long ld_a, const int* __restrict__ lens) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* tws = reinterpret_cast<float4*>(smraw);
  float* xs = reinterpret_cast<float*>(tws + L);
  load_tw(tws, tw, L);
  const int nb = L / 2 + 1;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int n_act = lens != nullptr ? min(n_in, max(0, __ldg(lens + row / rows_a))) : n_in;
    __syncthreads();  // the previous row's samples are no longer read
    for (int n = threadIdx.x; n < n_act; n += blockDim.x) xs[n] = __ldg(x + row * n_in + n);
    __syncthreads();
    const long long base = (row / rows_a) * ld_a + (row % rows_a);
    for (int l = threadIdx.x; l < nb; l += blockDim.x) {
      dacc re{0.f, 0.f}, im{0.f, 0.f};
      int m = 0;  // (n l) mod L
      for (int n = 0; n < n_act; ++n) {
        const float4 w = tws[m];
        acc_mac_f(re, xs[n], tw_re(w));
        acc_mac_f(im, xs[n], tw_im(w));
        m += l;
        if (m >= L) m -= L;
      }
      const dfl r = acc_get(re), i = acc_get(im);
      X[l * ld_l + base] = make_float2(r.hi, i.hi);
      X_lo[l * ld_l + base] = make_float2(r.lo, i.lo);
    }
  }
}

// First n_keep samples of the length-L real inverse DFT of bins X[0..L/2]
// (pairs), for thread-strided n:  x[n] = (1/L) (X_0 + (-1)^n X_{L/2}
//   + 2 sum_{0 < l < L/2} Re(X_l exp(2 pi i n l / L))),
// Re(X_l conj(W^{nl})) = Re X_l Re W + Im X_l Im W with W = tw[(n l) mod L].
// Xs[l] holds (re hi, re lo, im hi, im lo).
template <class Out>
__device__ __forceinline__ void df_irfft_head(const float4* Xs, const float4* tws, int L, int n_keep, Out out) {
  const int N = L / 2;
  const float inv_l = 1.f / static_cast<float>(L);  // a power of two: exact
  for (int n = threadIdx.x; n < n_keep; n += blockDim.x) {
    dacc s{0.f, 0.f};
    int m = n;  // (n l) mod L for l = 1
    for (int l = 1; l < N; ++l) {
      const float4 w = tws[m];
      const float4 xv = Xs[l];
      acc_mac(s, dfl{xv.x, xv.y}, tw_re(w));
      acc_mac(s, dfl{xv.z, xv.w}, tw_im(w));
      m += n;
      if (m >= L) m -= L;
    }
    dfl t = acc_get(s);
    t = {2.f * t.hi, 2.f * t.lo};
    t = df_add(t, dfl{Xs[0].x, Xs[0].y});
    const float sg = (n & 1) ? -1.f : 1.f;
    t = df_add(t, dfl{sg * Xs[N].x, sg * Xs[N].y});
    out(n, dfl{t.hi * inv_l, t.lo * inv_l});
  }
}

// Retransform of grid rows i (CTAs loop over them), pairs in and out:
//   mhat[l][i] -> IFFT, keep n < N -> m -> v = D_t m (backward difference, or
//   v = m) -> zero-pad to L, DFT -> vhat[l][i];  m optionally to seafloor[i][n]
// (rounded to FP32).  inv_dt as a pair.
__global__ void __launch_bounds__(kDfThreads) k_df_retransform(const float2* __restrict__ mhat,
                                                               const float2* __restrict__ mhat_lo, long long Ng,
                                                               long long ld_m, int L, const float4* __restrict__ tw,
                                                               float inv_dt_hi, float inv_dt_lo, int dt_mode,
                                                               float2* vhat, float2* vhat_lo, long long ld_v,
                                                               float* seafloor) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = L / 2;
  float4* tws = reinterpret_cast<float4*>(smraw);
  float4* Xs = tws + L;                                  // [N + 1]
  float2* ms = reinterpret_cast<float2*>(Xs + N + 1);    // [N] pairs (hi, lo)
  float2* vs = ms + N;                                   // [N]
  load_tw(tws, tw, L);
  const dfl inv_dt{inv_dt_hi, inv_dt_lo};
  for (long long i = blockIdx.x; i < Ng; i += gridDim.x) {
    __syncthreads();
    for (int l = threadIdx.x; l <= N; l += blockDim.x) {
      const float2 h = __ldg(mhat + l * ld_m + i), o = __ldg(mhat_lo + l * ld_m + i);
      Xs[l] = make_float4(h.x, o.x, h.y, o.y);
    }
    __syncthreads();
    df_irfft_head(Xs, tws, L, N, [&](int n, dfl v) {
      ms[n] = make_float2(v.hi, v.lo);
      if (seafloor != nullptr) seafloor[i * N + n] = v.hi + v.lo;
    });
    __syncthreads();
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
      const dfl m{ms[n].x, ms[n].y};
      dfl v = m;
      if (dt_mode != S2W_DT_NONE) {
        const dfl mp = n > 0 ? dfl{ms[n - 1].x, ms[n - 1].y} : dfl{0.f, 0.f};
        v = df_mul(df_add(m, df_neg(mp)), inv_dt);
      }
      vs[n] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    for (int l = threadIdx.x; l <= N; l += blockDim.x) {
      dacc re{0.f, 0.f}, im{0.f, 0.f};
      int m = 0;
      for (int n = 0; n < N; ++n) {
        const float4 w = tws[m];
        const dfl v{vs[n].x, vs[n].y};
        acc_mac(re, v, tw_re(w));
        acc_mac(im, v, tw_im(w));
        m += l;
        if (m >= L) m -= L;
      }
      const dfl r = acc_get(re), q = acc_get(im);
      vhat[l * ld_v + i] = make_float2(r.hi, q.hi);
      vhat_lo[l * ld_v + i] = make_float2(r.lo, q.lo);
    }
  }
}

// One CTA per (rupture b, observation o): Qhat[l] = sum over the nseg
// segment partials in fixed order (pairs), then q[b][o][n], n < n_keep, of
// the length-L inverse DFT (rounded to FP32), rows n_keep apart.
__global__ void __launch_bounds__(kDfThreads) k_df_reduce_irfft(const float2* __restrict__ part,
                                                                const float2* __restrict__ part_lo, int No, int nseg,
                                                                long long s_b, long long s_l, long long s_s, int L,
                                                                const float4* __restrict__ tw, float* q, int n_keep) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = L / 2;
  float4* tws = reinterpret_cast<float4*>(smraw);
  float4* Xs = tws + L;
  load_tw(tws, tw, L);
  const int b = blockIdx.x / No, o = blockIdx.x % No;
  const long long pb = b * s_b + o;
  for (int k = threadIdx.x; k <= N; k += blockDim.x) {
    dacc re{0.f, 0.f}, im{0.f, 0.f};
    for (int s = 0; s < nseg; ++s) {
      const long long e = pb + k * s_l + s * s_s;
      const float2 h = __ldg(part + e), lo = __ldg(part_lo + e);
      acc_add(re, dfl{h.x, lo.x});
      acc_add(im, dfl{h.y, lo.y});
    }
    const dfl r = acc_get(re), i = acc_get(im);
    Xs[k] = make_float4(r.hi, r.lo, i.hi, i.lo);
  }
  __syncthreads();
  float* out = q + static_cast<long long>(blockIdx.x) * n_keep;
  df_irfft_head(Xs, tws, L, n_keep, [&](int n, dfl v) { out[n] = v.hi + v.lo; });
}

unsigned df_grid(long long units) {
  long long g = units < 152LL * 8 ? units : 152LL * 8;
  return static_cast<unsigned>(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_twiddles_df(float4* tw, int L, cudaStream_t st) {
  k_twiddles_df<<<(L + 255) / 256, 256, 0, st>>>(tw, L);
  return cudaGetLastError();
}

cudaError_t launch_df_rfft_rows(const float* x, long long rows, int n_in, int Nt, const float4* tw, float2* X,
                                float2* X_lo, long long ld_l, long long rows_a, long long ld_a, cudaStream_t st,
                                const int* lens) {
  if (rows <= 0) return cudaSuccess;
  if (n_in < 1 || n_in > Nt || Nt < 1 || Nt > 512) return cudaErrorInvalidValue;
  const int L = 2 * Nt;
  const size_t sm = sizeof(float4) * L + sizeof(float) * Nt;
  k_df_rfft_rows<<<df_grid(rows), kDfThreads, sm, st>>>(x, rows, n_in, L, tw, X, X_lo, ld_l, rows_a, ld_a, lens);
  return cudaGetLastError();
}

cudaError_t launch_df_retransform(const float2* mhat, const float2* mhat_lo, long long Ng, long long ld_m, int Nt,
                                  const float4* tw, double inv_dt, int dt_mode, float2* vhat, float2* vhat_lo,
                                  long long ld_v, float* seafloor, cudaStream_t st) {
  if (Ng <= 0) return cudaSuccess;
  if (Nt < 1 || Nt > 512 || (dt_mode != S2W_DT_BACKWARD && dt_mode != S2W_DT_NONE)) return cudaErrorInvalidValue;
  const int L = 2 * Nt;
  const size_t sm = sizeof(float4) * (L + Nt + 1) + sizeof(float2) * 2 * Nt;
  const float ih = static_cast<float>(inv_dt);
  const float il = static_cast<float>(inv_dt - static_cast<double>(ih));
  k_df_retransform<<<df_grid(Ng), kDfThreads, sm, st>>>(mhat, mhat_lo, Ng, ld_m, L, tw, ih, il, dt_mode, vhat,
                                                         vhat_lo, ld_v, seafloor);
  return cudaGetLastError();
}

cudaError_t launch_df_reduce_irfft(const float2* part, const float2* part_lo, int B, int No, int nseg, int Nt,
                                   long long s_b, long long s_l, long long s_s, const float4* tw, float* q,
                                   cudaStream_t st, int n_keep) {
  if (n_keep <= 0 || n_keep > Nt) n_keep = Nt;
  const long long n = static_cast<long long>(B) * No;
  if (n <= 0) return cudaSuccess;
  if (Nt < 1 || Nt > 512) return cudaErrorInvalidValue;
  const int L = 2 * Nt;
  const size_t sm = sizeof(float4) * (L + Nt + 1);
  k_df_reduce_irfft<<<static_cast<unsigned>(n), kDfThreads, sm, st>>>(part, part_lo, No, nseg, s_b, s_l, s_s, L, tw,
                                                                      q, n_keep);
  return cudaGetLastError();
}

}  // namespace s2w
