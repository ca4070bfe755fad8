// Warp-level FFTs used by every transform in the pipeline (Alg. 2: ZeroPad
// then FFT, and IFFT then Truncate).
//
// One warp transforms one signal.  A complex DFT of N = 32 P points is split
// four-step style as N = P x 32: lane l holds z[l + 32 t] in register t;
//   (a) a P-point DFT over t in registers (radix-2, decimation in frequency),
//   (b) a twiddle W_N^(l k2),
//   (c) a 32-point DFT across lanes (five radix-2 stages on __shfl_xor_sync),
// after which lane l holds Z[k2 + P rev5(l)] in register k2.
//
// A real signal of length L = 2N is packed as z[n] = x[2n] + i x[2n+1]; the
// N + 1 bins of its real DFT follow from Z[k] and conj(Z[N - k]).  Twiddles
// come from a shared-memory table tw[m] = exp(-2 pi i m / L), m < L, whose
// entries are computed in FP64 once per context (k_fft.cu: k_twiddles).
#pragma once

#include "s2w_internal.cuh"

namespace s2w {

__device__ __forceinline__ int rev5(int l) { return static_cast<int>(__brev(static_cast<unsigned>(l)) >> 27); }

template <int P>
__host__ __device__ constexpr int bitrev_p(int k) {
  int r = 0;
  for (int b = 1; b < P; b <<= 1) {
    r <<= 1;
    if (k & b) r |= 1;
  }
  return r;
}

// Forward complex DFT of N = 32 P points (see file comment for layouts).
template <int P>
__device__ __forceinline__ void warp_fft(float2 (&v)[P], const float2* __restrict__ tw, int lane) {
  constexpr int N = 32 * P;
  constexpr int L = 2 * N;
  // (a) P-point DFT over registers; output position p holds bin bitrev(p).
#pragma unroll
  for (int h = P / 2; h >= 1; h >>= 1) {
#pragma unroll
    for (int b = 0; b < P; b += 2 * h) {
#pragma unroll
      for (int j = 0; j < h; ++j) {
        const float2 a = v[b + j];
        const float2 c = v[b + j + h];
        v[b + j] = cadd(a, c);
        v[b + j + h] = (j == 0) ? csub(a, c) : cmul(csub(a, c), tw[j * (L / (2 * h))]);
      }
    }
  }
  float2 y[P];
#pragma unroll
  for (int k = 0; k < P; ++k) y[k] = v[bitrev_p<P>(k)];
  // (b) twiddle W_N^(l k2) = W_L^(2 ((l k2) mod N))
#pragma unroll
  for (int k = 1; k < P; ++k) y[k] = cmul(y[k], tw[2 * ((lane * k) & (N - 1))]);
  // (c) 32-point DFT across lanes, decimation in frequency on the lane bits.
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
    const float2 w = tw[(lane & (h - 1)) * (L / (2 * h))];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      float2 p;
      p.x = __shfl_xor_sync(0xffffffffu, y[k].x, h);
      p.y = __shfl_xor_sync(0xffffffffu, y[k].y, h);
      y[k] = upper ? cmul(csub(p, y[k]), w) : cadd(y[k], p);
    }
  }
#pragma unroll
  for (int k = 0; k < P; ++k) v[k] = y[k];
}

// Forward real FFT, step 1: pack, transform, store Z[0..N) in natural order
// into the warp's shared scratch `zs`.  get(n) returns x[n] (0 past the end).
template <int P, class Get>
__device__ __forceinline__ void warp_rfft_stage(Get get, float2* zs, const float2* __restrict__ tw, int lane) {
  float2 v[P];
#pragma unroll
  for (int t = 0; t < P; ++t) {
    const int n = lane + 32 * t;
    v[t] = make_float2(get(2 * n), get(2 * n + 1));
  }
  warp_fft<P>(v, tw, lane);
  const int k1 = rev5(lane);
#pragma unroll
  for (int k = 0; k < P; ++k) zs[k + P * k1] = v[k];
  __syncwarp();
}

// Forward real FFT, step 2: bin k (0 <= k <= N) of the length-2N real DFT.
//   X[k] = E[k] + W_L^k O[k],  E = (Z[k] + conj Z[N-k]) / 2,
//   O = (Z[k] - conj Z[N-k]) / 2i,  with Z[N] = Z[0].
template <int P>
__device__ __forceinline__ float2 rfft_bin(const float2* zs, const float2* __restrict__ tw, int k) {
  constexpr int N = 32 * P;
  const float2 zk = zs[k & (N - 1)];
  const float2 zc = cconj(zs[(N - k) & (N - 1)]);
  const float2 e = cscale(cadd(zk, zc), 0.5f);
  const float2 d = csub(zk, zc);
  const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);
  return cadd(e, cmul(tw[k], o));
}

// Inverse real FFT with truncation: from the N + 1 bins X[0..N] of a real
// length-2N signal, produce its first N samples
//   x[n] = (1/L) sum_{k<L} X[k] W_L^(-n k),  n < N,
// handing each to put(n, value).  getx(k) returns X[k] for 0 <= k <= N.
template <int P, class GetX, class Put>
__device__ __forceinline__ void warp_irfft_head(GetX getx, Put put, const float2* __restrict__ tw, int lane) {
  constexpr int N = 32 * P;
  float2 v[P];
#pragma unroll
  for (int t = 0; t < P; ++t) {
    const int k = lane + 32 * t;
    const float2 xk = getx(k);
    const float2 xc = cconj(getx(N - k));
    const float2 e = cscale(cadd(xk, xc), 0.5f);
    const float2 o = cmul(cscale(csub(xk, xc), 0.5f), cconj(tw[k]));
    // Z = E + i O, fed to the forward transform conjugated (inverse by conjugation)
    v[t] = make_float2(e.x - o.y, -(e.y + o.x));
  }
  warp_fft<P>(v, tw, lane);
  const int k1 = rev5(lane);
  const float s = 1.0f / static_cast<float>(N);
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int n = k + P * k1;
    if (n < N / 2) {
      put(2 * n, v[k].x * s);
      put(2 * n + 1, -v[k].y * s);
    }
  }
}

}  // namespace s2w
