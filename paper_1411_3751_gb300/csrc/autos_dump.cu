// Total-power (autocorrelation) kernel and the dump/format kernel.
#include "corr_internal.cuh"

namespace corr {
namespace {

__device__ __forceinline__ int nib(unsigned v) { return ((int)(v & 0xF) ^ 8) - 8; }

__device__ __forceinline__ int power_of(unsigned b) {
  const int re = nib(b >> 4), im = nib(b);
  return re * re + im * im;
}

// Autocorrelations A[f][n] += sum_t |x_{f,n}(t)|^2 (Sec. 2.6: total power of selected inputs at a
// high cadence), and optionally the offset sums s[f][n] += sum_t (x + 8 + 8i) needed to map the
// tensor path's offset-domain products back to V (see the fused X-engine). One block of 4 warps per
// (channel, group of 32 inputs). Lane l of a warp reads the 4 inputs 4 (l % 8) .. +3 at time offset
// l / 8, so each warp covers 32 inputs x 4 samples per step and each sample byte is read once.
// Per-thread int32 partials are reduced over the four time lanes with warp shuffles, then over the
// 4 warps through shared memory, and added to int64.
constexpr int AW = 4;

__global__ void __launch_bounds__(AW * 32) autos_kernel(const uint8_t* __restrict__ in, int N, int C, int T,
                                                        long long* __restrict__ autos, long long* __restrict__ soff) {
  const int f = blockIdx.y;
  const int n0 = blockIdx.x * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane & 7, toff = lane >> 3;  // inputs n0 + 4 sub .. +3, time offset 0..3
  int acc[4] = {0, 0, 0, 0}, sr[4] = {0, 0, 0, 0}, si[4] = {0, 0, 0, 0};
  long long acc64[4] = {0, 0, 0, 0}, sr64[4] = {0, 0, 0, 0}, si64[4] = {0, 0, 0, 0};
  int since = 0;
  for (int t = warp * 4 + toff; t < T; t += AW * 4) {
    const uint8_t* row = in + ((size_t)t * C + f) * N + n0 + 4 * sub;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (n0 + 4 * sub + q < N) {
        const unsigned b = row[q];
        acc[q] += power_of(b);
        sr[q] += (int)((b >> 4) ^ 8u);   // Re + 8
        si[q] += (int)((b & 15u) ^ 8u);  // Im + 8
      }
    if (++since == (1 << 20)) {  // int32 partials stay below 128 * 2^20
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc64[q] += acc[q];
        sr64[q] += sr[q];
        si64[q] += si[q];
        acc[q] = sr[q] = si[q] = 0;
      }
      since = 0;
    }
  }
  __shared__ long long part[3][AW][32];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    long long v[3] = {acc64[q] + acc[q], sr64[q] + sr[q], si64[q] + si[q]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v[k] += __shfl_xor_sync(0xffffffffu, v[k], 8);
      v[k] += __shfl_xor_sync(0xffffffffu, v[k], 16);
      if (toff == 0) part[k][warp][4 * sub + q] = v[k];
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int n = n0 + threadIdx.x;
    long long sum[3] = {0, 0, 0};
#pragma unroll
    for (int w = 0; w < AW; ++w)
#pragma unroll
      for (int k = 0; k < 3; ++k) sum[k] += part[k][w][threadIdx.x];
    if (n < N) {
      autos[(long long)f * N + n] += sum[0];
      if (soff) {
        soff[((long long)f * N + n) * 2] += sum[1];
        soff[((long long)f * N + n) * 2 + 1] += sum[2];
      }
    }
  }
}

// Dump: out[k] = fmt(acc[k]). CI64 copies, CF32 rounds to nearest float, CF32_NORM divides by the
// sample count in double and rounds to float. Contributions of the tensor path are held in the
// offset domain (u = x + 8 + 8i) and are mapped back here:
//   V = Vu - (8 - 8i) s_a - (8 + 8i) conj(s_c) + 128 T_off,   A = Au - 16 (Re s + Im s) + 128 T_off
// (s = per-input offset sums and T_off = samples accumulated through that path, per cadence).
template <typename T>
__device__ __forceinline__ void put(void* out, long long k, long long v, int fmt, long long n_samples) {
  if (fmt == CORR_FMT_CI64) {
    static_cast<long long*>(out)[k] = v;
  } else if (fmt == CORR_FMT_CF32) {
    static_cast<float*>(out)[k] = __ll2float_rn(v);
  } else {
    static_cast<float*>(out)[k] = n_samples > 0 ? __double2float_rn(__ddiv_rn(__ll2double_rn(v), (double)n_samples)) : 0.f;
  }
}

// station pair index b -> (a, c) with b = a (a + 1) / 2 + c, a >= c
__device__ __forceinline__ void pair_of(int b, int& sa, int& sc) {
  int a = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
  while ((long long)a * (a + 1) / 2 > b) --a;
  while ((long long)(a + 1) * (a + 2) / 2 <= b) ++a;
  sa = a;
  sc = b - (int)((long long)a * (a + 1) / 2);
}

// Corrected value of cross cell `cell` (= f * B_s * P + b * P + pidx) from its raw int64 sums.
__device__ __forceinline__ void cross_value(const long long* __restrict__ acc, long long cell, long long f, int b,
                                            int pidx, const Shape2& g, long long& re, long long& im) {
  const longlong2 v2 = reinterpret_cast<const longlong2*>(acc)[cell];
  re = v2.x;
  im = v2.y;
  if (g.soff != nullptr && g.t_off != 0) {
    int sa, sc;
    pair_of(b, sa, sc);
    const long long a = (long long)sa * g.npol + pidx / g.npol;
    const long long c = (long long)sc * g.npol + pidx % g.npol;
    const longlong2 s_a = reinterpret_cast<const longlong2*>(g.soff)[f * g.N + a];
    const longlong2 s_c = reinterpret_cast<const longlong2*>(g.soff)[f * g.N + c];
    re += -8 * (s_a.x + s_a.y + s_c.x + s_c.y) + 128 * g.t_off;
    im += -8 * (s_a.y - s_a.x + s_c.x - s_c.y);
  }
}

__device__ __forceinline__ long long auto_value(const long long* __restrict__ acc, long long k, const Shape2& g) {
  long long v = acc[k];
  if (g.soff != nullptr && g.t_off != 0) {
    const longlong2 s = reinterpret_cast<const longlong2*>(g.soff)[k];
    v += -16 * (s.x + s.y) + 128 * g.t_off;  // A = Au - 16 (Re s + Im s) + 128 T
  }
  return v;
}

// Cross dump of cells [cell0, cell0 + n_cells) (a cell = one (re, im) pair), output indexed from 0.
__global__ void dump_cross_kernel(const long long* __restrict__ acc, long long cell0, long long n_cells,
                                  void* __restrict__ out, int fmt, long long n_samples, Shape2 g) {
  const long long cpc = g.Bs * g.P;  // cells per channel
  const int lp = g.P == 4 ? 2 : 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_cells; k += (long long)gridDim.x * blockDim.x) {
    const long long cell = cell0 + k;
    const long long f = cell / cpc;
    const int r = (int)(cell - f * cpc);
    const int b = r >> lp, pidx = r & (g.P - 1);
    long long re, im;
    cross_value(acc, cell, f, b, pidx, g, re, im);
    const long long ns = g.base ? n_samples - g.base[b] : n_samples;
    put<void>(out, 2 * k, re, fmt, ns);
    put<void>(out, 2 * k + 1, im, fmt, ns);
  }
}

// Autos dump of elements [k0, k0 + n).
__global__ void dump_autos_kernel(const long long* __restrict__ acc, long long k0, long long n, void* __restrict__ out,
                                  int fmt, long long n_samples, Shape2 g) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long v = auto_value(acc, k0 + k, g);
    const long long ns = g.base ? n_samples - g.base[(k0 + k) % g.N] : n_samples;
    put<void>(out, k, v, fmt, ns);
  }
}

// Selective dump (Sec. 2.6: selected cells are dumped and zeroed at their own cadence). Cross: unit =
// (channel, list pair k >= l, product p q) -> sum x_{st[k] p} conj(x_{st[l] q}); the stored cell is
// (st[k] p, st[l] q) when st[k] >= st[l], else its conjugate (st[l] q, st[k] p). Autos: unit =
// (channel, list position k, pol p) -> input st[k] n_pol + p. A reset stores minus the corrected
// value's offset-domain correction, acc := acc - value, so the corrected value restarts from zero
// while the shared offset sums keep integrating (the correction is affine in them).
__global__ void dump_select_kernel(long long* __restrict__ acc, const int* __restrict__ st, int n_st, int f0, int nf,
                                   void* __restrict__ out, int fmt, long long n_samples, int reset, Shape2 g) {
  if (g.autos) {
    const long long per = (long long)n_st * g.npol;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < (long long)nf * per;
         u += (long long)gridDim.x * blockDim.x) {
      const long long fl = u / per;
      const int r = (int)(u - fl * per);
      const int i = st[r / g.npol] * g.npol + r % g.npol;
      const long long k = (f0 + fl) * g.N + i;
      const long long v = auto_value(acc, k, g);
      put<void>(out, u, v, fmt, g.base ? n_samples - g.base[i] : n_samples);
      if (reset) acc[k] -= v;
    }
    return;
  }
  const long long npairs = (long long)n_st * (n_st + 1) / 2;
  const long long per = npairs * g.P;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < (long long)nf * per;
       u += (long long)gridDim.x * blockDim.x) {
    const long long fl = u / per;
    const int r = (int)(u - fl * per);
    const int pr = r / g.P, pidx = r % g.P;
    int k, l;
    pair_of(pr, k, l);
    const int a = st[k], c = st[l], p = pidx / g.npol, q = pidx % g.npol;
    const bool swap = a < c;
    const int sa = swap ? c : a, sc = swap ? a : c;
    const int sp = swap ? q * g.npol + p : pidx;  // stored product index
    const int b = sa * (sa + 1) / 2 + sc;
    const long long f = f0 + fl;
    const long long cell = (f * g.Bs + b) * g.P + sp;
    long long re, im;
    cross_value(acc, cell, f, b, sp, g, re, im);
    const long long ns = g.base ? n_samples - g.base[b] : n_samples;
    put<void>(out, 2 * u, re, fmt, ns);
    put<void>(out, 2 * u + 1, swap ? -im : im, fmt, ns);
    if (reset) {
      acc[2 * cell] -= re;
      acc[2 * cell + 1] -= im;
    }
  }
}

__global__ void set_base_kernel(long long* __restrict__ base, const int* __restrict__ st, int n_st, long long value,
                                int npol, int autos) {
  const long long n = autos ? (long long)n_st * npol : (long long)n_st * (n_st + 1) / 2;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
    if (autos) {
      base[st[u / npol] * npol + u % npol] = value;
    } else {
      int k, l;
      pair_of((int)u, k, l);
      const int a = st[k] > st[l] ? st[k] : st[l], c = st[k] > st[l] ? st[l] : st[k];
      base[a * (a + 1) / 2 + c] = value;
    }
  }
}

}  // namespace

cudaError_t launch_autos(const Shape& s, const uint8_t* d_in, int T_blk, long long* d_autos, long long* d_soff,
                         cudaStream_t st) {
  if (T_blk == 0) return cudaSuccess;
  dim3 grid((s.N + 31) / 32, s.C);
  autos_kernel<<<grid, AW * 32, 0, st>>>(d_in, s.N, s.C, T_blk, d_autos, d_soff);
  return cudaGetLastError();
}

cudaError_t launch_dump_select(long long* d_acc, const int* d_st, int n_st, int f0, int nf, void* d_out, int fmt,
                               long long n_samples, int reset, const Shape2& g, cudaStream_t st) {
  const long long units = (long long)nf * (g.autos ? (long long)n_st * g.npol : (long long)n_st * (n_st + 1) / 2 * g.P);
  if (units == 0) return cudaSuccess;
  long long blocks = (units + 255) / 256;
  if (blocks > (long long)sm_count() * 32) blocks = (long long)sm_count() * 32;
  dump_select_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_acc, d_st, n_st, f0, nf, d_out, fmt, n_samples, reset, g);
  return cudaGetLastError();
}

cudaError_t launch_set_base(long long* d_base, const int* d_st, int n_st, long long value, const Shape2& g,
                            cudaStream_t st) {
  const long long n = g.autos ? (long long)n_st * g.npol : (long long)n_st * (n_st + 1) / 2;
  long long blocks = (n + 255) / 256;
  if (blocks > (long long)sm_count() * 8) blocks = (long long)sm_count() * 8;
  if (blocks == 0) return cudaSuccess;
  set_base_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_base, d_st, n_st, value, g.npol, g.autos);
  return cudaGetLastError();
}

cudaError_t launch_dump(const long long* d_acc, long long n_elems, void* d_out, int fmt, long long n_samples,
                        long long k_base, const Shape2& g, cudaStream_t st) {
  if (n_elems == 0) return cudaSuccess;
  const long long n_units = g.autos ? n_elems : n_elems / 2;
  long long blocks = (n_units + 255) / 256;
  if (blocks > (long long)sm_count() * 32) blocks = (long long)sm_count() * 32;
  if (g.autos)
    dump_autos_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_acc, k_base, n_elems, d_out, fmt, n_samples, g);
  else
    dump_cross_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_acc, k_base / 2, n_elems / 2, d_out, fmt, n_samples, g);
  return cudaGetLastError();
}

}  // namespace corr
