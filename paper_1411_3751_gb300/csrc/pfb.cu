// Polyphase filterbank (PFB) F-engine (Sec. 2.2): each input's real 8-bit ADC stream is split into
// frames of M = 8192 samples; spectrum t weights the P = n_taps frames t .. t + P - 1 by the
// prototype filter (FIR, exact in integers: 8-bit samples x 18-bit coefficients), sums them, and
// takes an M-point real DFT, keeping channels 0 .. M/2 - 1 (24.0 kHz apart at a 196.608 MHz clock).
// The paper's fixed-point FFT halves at each of its log2(M) = 13 stages; here the FFT runs in FP32
// and the result is scaled by the same 2^-13 once (an exact power of two).
//
//   y_t[m] = sum_p h[p M + m] x[(t + p) M + m]                       (int32, exact)
//   X_t[k] = 2^-13 sum_m y_t[m] exp(-2 pi i k m / M),  k < M / 2      (FP32)
//
// One CTA of 256 threads per (input, two spectra). The real DFT is a 4096-point complex FFT of
// z[j] = y[2j] + i y[2j+1] followed by the split step that separates the even and odd halves:
//   X[k] = (Z[k] + conj Z[-k]) / 2 - i W^k (Z[k] - conj Z[-k]) / 2,  W = exp(-2 pi i / M).
// The complex FFT is a Stockham autosort FFT (no bit reversal), three radix-16 passes in shared
// memory; each thread holds 16 points per pass. Twiddles come from tables computed on the host in
// double precision.
#include "corr_internal.cuh"

#include <cmath>
#include <mutex>

namespace corr {
namespace {

constexpr int PFB_M = 8192;          // real FFT length
constexpr int PFB_H = PFB_M / 2;     // complex FFT length / output channels
constexpr int PFB_NT = 256;
constexpr float PFB_SCALE = 1.0f / 8192.0f;  // 2^-13

__device__ float2 g_w4096[PFB_H];  // exp(-2 pi i j / 4096)
__device__ float2 g_w8192[PFB_H];  // exp(-2 pi i k / 8192), k < 4096

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // a * (-i)

// shared-memory index with one pad element per 16 (breaks the stride-16 bank pattern of pass 0)
__device__ __forceinline__ int sidx(int i) { return i + (i >> 4); }

// In-register forward 16-point DFT, X[q] = sum_r v[r] exp(-2 pi i r q / 16), as 4 x 4: 4-point DFTs
// over a (r = 4 a + b), twiddles exp(-2 pi i b k1 / 16), 4-point DFTs over b; output X[k1 + 4 k2].
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = mul_mi(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

__device__ __forceinline__ void dft16(float2 (&v)[16]) {
  constexpr float C1 = 0.92387953251128674f;  // cos(pi / 8)
  constexpr float S1 = 0.38268343236508978f;  // sin(pi / 8)
  constexpr float R2 = 0.70710678118654752f;  // cos(pi / 4)
#pragma unroll
  for (int b = 0; b < 4; ++b) dft4(v[b], v[b + 4], v[b + 8], v[b + 12]);  // now v[4 k1 + b] = A[b][k1]
  // twiddles exp(-2 pi i b k1 / 16) for b, k1 in 1..3
  v[5] = cmul(v[5], make_float2(C1, -S1));    // b=1,k1=1: m=1
  v[9] = cmul(v[9], make_float2(R2, -R2));    // b=1,k1=2: m=2
  v[13] = cmul(v[13], make_float2(S1, -C1));  // b=1,k1=3: m=3
  v[6] = cmul(v[6], make_float2(R2, -R2));    // b=2,k1=1: m=2
  v[10] = mul_mi(v[10]);                      // b=2,k1=2: m=4
  v[14] = cmul(v[14], make_float2(-R2, -R2)); // b=2,k1=3: m=6
  v[7] = cmul(v[7], make_float2(S1, -C1));    // b=3,k1=1: m=3
  v[11] = cmul(v[11], make_float2(-R2, -R2)); // b=3,k1=2: m=6
  v[15] = cmul(v[15], make_float2(-C1, S1));  // b=3,k1=3: m=9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // now v[4 k1 + k2] = X[k1 + 4 k2]; reorder to natural order
  float2 t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = t[q];
}

constexpr int PFB_SPB = 2;                  // spectra per block (share the coefficient loads)
constexpr int PFB_ZLEN = PFB_H + PFB_H / 16;  // padded complex buffer per spectrum

// 4096-point complex FFT of z (padded layout) in place, Stockham radix 16: spans Ns = 1, 16, 256.
// The 15 twiddles exp(-2 pi i r k / (16 Ns)) of a thread come from 4 table loads, w^{4a+b} = w^{4a} w^b.
__device__ __forceinline__ void fft4096(float2* z, int tid) {
#pragma unroll 1
  for (int Ns = 1, tw = PFB_H / 16; Ns < PFB_H; Ns *= 16, tw /= 16) {
    const int k = tid & (Ns - 1);
    const int e = k * tw;  // < 4096 / 16; the table loads go out before the shared-memory loads
    float2 w1 = make_float2(1.f, 0.f), w4 = w1, w8 = w1, w12 = w1;
    if (Ns > 1) {
      w1 = g_w4096[e];
      w4 = g_w4096[4 * e];
      w8 = g_w4096[8 * e];
      w12 = g_w4096[12 * e];
    }
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = z[sidx(tid + r * (PFB_H / 16))];
    if (Ns > 1) {
      const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
      v[1] = cmul(v[1], w1);
      v[2] = cmul(v[2], w2);
      v[3] = cmul(v[3], w3);
      v[4] = cmul(v[4], w4);
      v[5] = cmul(v[5], cmul(w4, w1));
      v[6] = cmul(v[6], cmul(w4, w2));
      v[7] = cmul(v[7], cmul(w4, w3));
      v[8] = cmul(v[8], w8);
      v[9] = cmul(v[9], cmul(w8, w1));
      v[10] = cmul(v[10], cmul(w8, w2));
      v[11] = cmul(v[11], cmul(w8, w3));
      v[12] = cmul(v[12], w12);
      v[13] = cmul(v[13], cmul(w12, w1));
      v[14] = cmul(v[14], cmul(w12, w2));
      v[15] = cmul(v[15], cmul(w12, w3));
    }
    dft16(v);
    __syncthreads();
    const int base = (tid - k) * 16 + k;
#pragma unroll
    for (int q = 0; q < 16; ++q) z[sidx(base + q * Ns)] = v[q];
    __syncthreads();
  }
}

// Split step: X[k] from Z[k] and Z[4096 - k], scaled, written to o[0 .. 4095].
__device__ __forceinline__ void split_store(const float2* z, float2* __restrict__ o, int tid) {
  if (tid == 0) {
    const float2 z0 = z[sidx(0)];
    o[0] = make_float2((z0.x + z0.y) * PFB_SCALE, 0.f);  // DC; the Nyquist bin (z0.x - z0.y) is not kept
    const float2 zh = z[sidx(PFB_H / 2)];              // k = 2048: X = conj(Z[2048]) (W^2048 = -i)
    o[PFB_H / 2] = make_float2(zh.x * PFB_SCALE, -zh.y * PFB_SCALE);
  }
  float2 wk[PFB_H / 2 / PFB_NT];  // this thread's split twiddles, loaded together
#pragma unroll
  for (int q = 0; q < PFB_H / 2 / PFB_NT; ++q) {
    const int k = 1 + tid + q * PFB_NT;
    wk[q] = k < PFB_H / 2 ? g_w8192[k] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int q = 0; q < PFB_H / 2 / PFB_NT; ++q) {
    const int k = 1 + tid + q * PFB_NT;
    if (k >= PFB_H / 2) break;
    const float2 a = z[sidx(k)], b = z[sidx(PFB_H - k)];
    const float2 w = wk[q];
    const float2 wm = make_float2(-w.x, w.y);  // W^(4096 - k) = -conj(W^k)
    // k: E = (a + conj b) / 2, O = (a - conj b) / 2, X[k] = E - i W^k O
    {
      const float2 e = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
      const float2 od = make_float2(0.5f * (a.x - b.x), 0.5f * (a.y + b.y));
      const float2 wo = mul_mi(cmul(w, od));
      o[k] = make_float2((e.x + wo.x) * PFB_SCALE, (e.y + wo.y) * PFB_SCALE);
    }
    // 4096 - k: roles of a and b swap
    {
      const float2 e = make_float2(0.5f * (b.x + a.x), 0.5f * (b.y - a.y));
      const float2 od = make_float2(0.5f * (b.x - a.x), 0.5f * (b.y + a.y));
      const float2 wo = mul_mi(cmul(wm, od));
      o[PFB_H - k] = make_float2((e.x + wo.x) * PFB_SCALE, (e.y + wo.y) * PFB_SCALE);
    }
  }
}

// 8 samples of one frame at p (8-byte aligned when vec8, else 4-byte aligned), as two words.
__device__ __forceinline__ int2 load8(const int8_t* __restrict__ p, bool vec8) {
  if (vec8) return __ldg(reinterpret_cast<const int2*>(p));
  return make_int2(__ldg(reinterpret_cast<const int*>(p)), __ldg(reinterpret_cast<const int*>(p) + 1));
}
__device__ __forceinline__ int sbyte(int2 w, int k) {  // signed byte k (0..7) of w
  const int v = k < 4 ? w.x : w.y;
  return (int)(int8_t)(uint8_t)((unsigned)v >> (8 * (k & 3)));
}
__device__ __forceinline__ void fir_tap(int (&y)[8], const int4& c0, const int4& c1, int2 xs) {
  y[0] += c0.x * sbyte(xs, 0);
  y[1] += c0.y * sbyte(xs, 1);
  y[2] += c0.z * sbyte(xs, 2);
  y[3] += c0.w * sbyte(xs, 3);
  y[4] += c1.x * sbyte(xs, 4);
  y[5] += c1.y * sbyte(xs, 5);
  y[6] += c1.z * sbyte(xs, 6);
  y[7] += c1.w * sbyte(xs, 7);
}

// One CTA per (input, pair of spectra t0, t0 + 1): the FIR of both spectra shares each coefficient
// load and each frame load (frames t0 .. t0 + P), then each spectrum is transformed in its own shared
// buffer. PT > 0 fixes the tap count at compile time (all loads of a step issued together); PT == 0
// takes it from P.
template <int PT>
__global__ void __launch_bounds__(PFB_NT, 3) pfb_kernel(const int8_t* __restrict__ adc, long long stride, int T,
                                                        int P, bool vec8, const int* __restrict__ h,
                                                        float2* __restrict__ out) {
  extern __shared__ float2 zs[];  // PFB_SPB buffers of PFB_ZLEN
  const int t0 = blockIdx.x * PFB_SPB, n = blockIdx.y, tid = threadIdx.x;
  const int ns = T - t0 < PFB_SPB ? T - t0 : PFB_SPB;
  const int8_t* x = adc + (size_t)n * stride + (size_t)t0 * PFB_M;
  // FIR: thread handles samples m = 8 tid + 2048 j .. + 7 (j < 4), for both spectra
#pragma unroll 1
  for (int j = 0; j < PFB_M / (8 * PFB_NT); ++j) {
    const int m = 8 * tid + 8 * PFB_NT * j;
    int y[PFB_SPB][8];
#pragma unroll
    for (int s = 0; s < PFB_SPB; ++s)
#pragma unroll
      for (int k = 0; k < 8; ++k) y[s][k] = 0;
    if (PT > 0) {
      int2 fr[PT + 1];  // frames t0 .. t0 + PT at m
#pragma unroll
      for (int q = 0; q <= PT; ++q) fr[q] = q < PT || ns > 1 ? load8(x + (size_t)q * PFB_M + m, vec8) : make_int2(0, 0);
#pragma unroll
      for (int p = 0; p < PT; ++p) {
        const int4* hp = reinterpret_cast<const int4*>(h + p * PFB_M + m);
        const int4 c0 = __ldg(hp), c1 = __ldg(hp + 1);
        fir_tap(y[0], c0, c1, fr[p]);
        fir_tap(y[1], c0, c1, fr[p + 1]);
      }
    } else {
#pragma unroll 2
      for (int p = 0; p < P; ++p) {
        const int4* hp = reinterpret_cast<const int4*>(h + p * PFB_M + m);
        const int4 c0 = __ldg(hp), c1 = __ldg(hp + 1);
        fir_tap(y[0], c0, c1, load8(x + (size_t)p * PFB_M + m, vec8));
        if (ns > 1) fir_tap(y[1], c0, c1, load8(x + (size_t)(p + 1) * PFB_M + m, vec8));
      }
    }
#pragma unroll
    for (int s = 0; s < PFB_SPB; ++s)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        zs[s * PFB_ZLEN + sidx(m / 2 + q)] = make_float2((float)y[s][2 * q], (float)y[s][2 * q + 1]);
  }
  __syncthreads();
  for (int s = 0; s < ns; ++s) {
    fft4096(zs + s * PFB_ZLEN, tid);
    split_store(zs + s * PFB_ZLEN, out + ((size_t)n * T + t0 + s) * PFB_H, tid);
  }
}

std::once_flag g_tw_once[64];
cudaError_t g_tw_err[64];

cudaError_t ensure_twiddles(int dev) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::call_once(g_tw_once[dev], [dev]() {
    float2 w1[PFB_H], w2[PFB_H];
    for (int j = 0; j < PFB_H; ++j) {
      const double a1 = -2.0 * M_PI * j / 4096.0, a2 = -2.0 * M_PI * j / 8192.0;
      w1[j] = make_float2((float)std::cos(a1), (float)std::sin(a1));
      w2[j] = make_float2((float)std::cos(a2), (float)std::sin(a2));
    }
    cudaError_t e = cudaMemcpyToSymbol(g_w4096, w1, sizeof(w1));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_w8192, w2, sizeof(w2));
    g_tw_err[dev] = e;
  });
  return g_tw_err[dev];
}

}  // namespace

cudaError_t launch_pfb(const int8_t* d_adc, long long stride, int N, int T, int P, const int* d_h, float2* d_out,
                       cudaStream_t st) {
  if ((long long)N * T == 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = ensure_twiddles(dev);
  if (e != cudaSuccess) return e;
  constexpr int smem = PFB_SPB * PFB_ZLEN * (int)sizeof(float2);
  const bool vec8 = ((reinterpret_cast<uintptr_t>(d_adc) | (uintptr_t)stride) & 7) == 0;
  const dim3 grid((unsigned)((T + PFB_SPB - 1) / PFB_SPB), (unsigned)N);
  if (P == 4) {
    e = set_smem_limit(reinterpret_cast<const void*>(pfb_kernel<4>), smem);
    if (e != cudaSuccess) return e;
    pfb_kernel<4><<<grid, PFB_NT, smem, st>>>(d_adc, stride, T, P, vec8, d_h, d_out);
  } else {
    e = set_smem_limit(reinterpret_cast<const void*>(pfb_kernel<0>), smem);
    if (e != cudaSuccess) return e;
    pfb_kernel<0><<<grid, PFB_NT, smem, st>>>(d_adc, stride, T, P, vec8, d_h, d_out);
  }
  return cudaGetLastError();
}

}  // namespace corr
