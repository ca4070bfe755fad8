// Warp-level FFTs used by every transform in the pipeline (Alg. 2: ZeroPad
// then FFT, and IFFT then Truncate).
//
// One warp transforms one signal.  A complex DFT of N = 32 P points is split
// four-step style as N = P x 32: lane l holds z[l + 32 t] in register t;
//   (a) a P-point DFT over t in registers (radix-2, decimation in frequency),
//   (b) a twiddle W_N^(l k2),
//   (c) the P independent 32-point DFTs over the lanes.  With P = 1 they run
//       as five radix-2 stages on __shfl_xor_sync.  Otherwise one transpose
//       through the warp's shared scratch gives each group of Q = 32 / P
//       lanes one of them (lane q of group g holds the points q + Q j), and
//       it splits again as 32 = P x Q: a P-point DFT over j in registers, a
//       twiddle W_32^(q a), and a Q-point DFT across the group's lanes on
//       log2(Q) shuffle stages.
// fft_out<P>(lane, k) is the output bin that register k of `lane` holds.
//
// A real signal of length L = 2N is packed as z[n] = x[2n] + i x[2n+1]; the
// N + 1 bins of its real DFT follow from Z[k] and conj(Z[N - k]).  Twiddles
// come from a shared-memory table tw[m] = exp(-2 pi i m / L), m < L, whose
// entries are computed in FP64 once per context (k_fft.cu: k_twiddles); the
// per-lane ones are read once per warp into registers (FftLane).
#pragma once

#include "s2w_internal.cuh"

namespace s2w {

__device__ __forceinline__ int rev5(int l) { return static_cast<int>(__brev(static_cast<unsigned>(l)) >> 27); }

// Position of Z[i] in the per-warp scratch: XOR swizzle inside blocks of 16
// complex entries, so that the scatter of the transform's outputs and the
// natural-order reads of rfft_bin spread over the shared-memory banks.
__device__ __forceinline__ int zsw(int i) { return i ^ ((i >> 4) & 15); }

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }

template <int P>
__host__ __device__ constexpr int bitrev_p(int k) {
  int r = 0;
  for (int b = 1; b < P; b <<= 1) {
    r <<= 1;
    if (k & b) r |= 1;
  }
  return r;
}

// Output bin held by register k of `lane` after warp_fft<P>.
template <int P>
__device__ __forceinline__ int fft_out(int lane, int k) {
  if (P == 1) return rev5(lane);
  constexpr int Q = 32 / P;
  constexpr int LQ = ilog2c(Q);
  const int g = lane / Q, q = lane % Q;
  const int rq = LQ > 0 ? static_cast<int>(__brev(static_cast<unsigned>(q)) >> (32 - LQ)) : 0;
  return g + P * k + P * P * rq;
}

// Per-lane twiddles of warp_fft<P>, read once per warp.
template <int P>
struct FftLane {
  static constexpr int Q = 32 / P;
  static constexpr int NST = P == 1 ? 5 : ilog2c(Q);  // cross-lane radix-2 stages
  float2 tl[P];                        // W_N^(lane k)
  float2 tq[P];                        // W_32^(q a)
  float2 tc[NST > 0 ? NST : 1];        // stage twiddles of the cross-lane DFT
};

template <int P>
__device__ __forceinline__ FftLane<P> fft_lane(const float2* __restrict__ tw, int lane) {
  constexpr int N = 32 * P;
  constexpr int L = 2 * N;
  constexpr int Q = 32 / P;
  FftLane<P> f;
#pragma unroll
  for (int k = 0; k < P; ++k) f.tl[k] = tw[2 * ((lane * k) & (N - 1))];
  if (P == 1) {
#pragma unroll
    for (int st = 0; st < FftLane<P>::NST; ++st) {
      const int h = 16 >> st;
      f.tc[st] = tw[(lane & (h - 1)) * (L / (2 * h))];
    }
  } else {
    const int q = lane % Q;
#pragma unroll
    for (int a = 0; a < P; ++a) f.tq[a] = tw[((q * a) & 31) * (L / 32)];
#pragma unroll
    for (int st = 0; st < FftLane<P>::NST; ++st) {
      const int h = (Q / 2) >> st;
      f.tc[st] = tw[(q & (h - 1)) * (L / (2 * h))];
    }
  }
  return f;
}

// P-point DFT over registers (radix-2 DIF, uniform twiddles W_P^j = W_L^(j L / P)
// of the length-L table), result in natural order.
template <int P>
__device__ __forceinline__ void reg_dft(float2 (&v)[P], const float2* __restrict__ tw) {
  constexpr int L = 64 * P;
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
#pragma unroll
  for (int k = 0; k < P; ++k) v[k] = y[k];
}

// Forward complex DFT of N = 32 P points (see file comment for layouts);
// scr: the warp's shared scratch of N complex entries (unused for P = 1).
template <int P>
__device__ __forceinline__ void warp_fft(float2 (&v)[P], const float2* __restrict__ tw, const FftLane<P>& fl,
                                         int lane, float2* scr) {
  // (a) + (b)
  reg_dft<P>(v, tw);
#pragma unroll
  for (int k = 1; k < P; ++k) v[k] = cmul(v[k], fl.tl[k]);
  if (P == 1) {
    // (c) 32-point DFT across lanes, decimation in frequency on the lane bits
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int h = 16 >> st;
      const bool upper = (lane & h) != 0;
      float2 p;
      p.x = __shfl_xor_sync(0xffffffffu, v[0].x, h);
      p.y = __shfl_xor_sync(0xffffffffu, v[0].y, h);
      v[0] = upper ? cmul(csub(p, v[0]), fl.tc[st]) : cadd(v[0], p);
    }
    return;
  }
  constexpr int Q = 32 / P;
  const int g = lane / Q, q = lane % Q;
  // (c) transpose: row k2 of the scratch holds the 32 points of DFT k2
  // (column XOR (Q k2) keeps the group reads below on distinct banks)
  __syncwarp();
#pragma unroll
  for (int k = 0; k < P; ++k) scr[k * 32 + (lane ^ ((Q * k) & 31))] = v[k];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < P; ++j) v[j] = scr[g * 32 + ((q + Q * j) ^ ((Q * g) & 31))];
  __syncwarp();
  reg_dft<P>(v, tw);
#pragma unroll
  for (int a = 1; a < P; ++a) v[a] = cmul(v[a], fl.tq[a]);
#pragma unroll
  for (int st = 0; st < FftLane<P>::NST; ++st) {
    const int h = (Q / 2) >> st;
    const bool upper = (q & h) != 0;
#pragma unroll
    for (int a = 0; a < P; ++a) {
      float2 p;
      p.x = __shfl_xor_sync(0xffffffffu, v[a].x, h);
      p.y = __shfl_xor_sync(0xffffffffu, v[a].y, h);
      v[a] = upper ? cmul(csub(p, v[a]), fl.tc[st]) : cadd(v[a], p);
    }
  }
}

// Forward real FFT, step 1: pack, transform, store Z[0..N) into the warp's
// shared scratch `zs` (Z[i] at zs[zsw(i)]).  get(n) returns x[n] (0 past the
// end).
template <int P, class Get>
__device__ __forceinline__ void warp_rfft_stage(Get get, float2* zs, const float2* __restrict__ tw,
                                                const FftLane<P>& fl, int lane) {
  float2 v[P];
#pragma unroll
  for (int t = 0; t < P; ++t) {
    const int n = lane + 32 * t;
    v[t] = make_float2(get(2 * n), get(2 * n + 1));
  }
  warp_fft<P>(v, tw, fl, lane, zs);
#pragma unroll
  for (int k = 0; k < P; ++k) zs[zsw(fft_out<P>(lane, k))] = v[k];
  __syncwarp();
}

// Forward real FFT, step 2: bin k (0 <= k <= N) of the length-2N real DFT.
//   X[k] = E[k] + W_L^k O[k],  E = (Z[k] + conj Z[N-k]) / 2,
//   O = (Z[k] - conj Z[N-k]) / 2i,  with Z[N] = Z[0].
template <int P>
__device__ __forceinline__ float2 rfft_bin(const float2* zs, const float2* __restrict__ tw, int k) {
  constexpr int N = 32 * P;
  const float2 zk = zs[zsw(k & (N - 1))];
  const float2 zc = cconj(zs[zsw((N - k) & (N - 1))]);
  const float2 e = cscale(cadd(zk, zc), 0.5f);
  const float2 d = csub(zk, zc);
  const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);
  return cadd(e, cmul(tw[k], o));
}

// Inverse real FFT with truncation: from the N + 1 bins X[0..N] of a real
// length-2N signal, produce its first N samples
//   x[n] = (1/L) sum_{k<L} X[k] W_L^(-n k),  n < N,
// handing each to put(n, value).  getx(k) returns X[k] for 0 <= k <= N; scr
// is the warp's shared scratch of N complex entries.
template <int P, class GetX, class Put>
__device__ __forceinline__ void warp_irfft_head(GetX getx, Put put, const float2* __restrict__ tw,
                                                const FftLane<P>& fl, int lane, float2* scr) {
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
  warp_fft<P>(v, tw, fl, lane, scr);
  const float s = 1.0f / static_cast<float>(N);
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int n = fft_out<P>(lane, k);
    if (n < N / 2) {
      put(2 * n, v[k].x * s);
      put(2 * n + 1, -v[k].y * s);
    }
  }
}

}  // namespace s2w
