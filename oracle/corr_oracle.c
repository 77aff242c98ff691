/*
 * CPU oracle for the X-engine (cross-multiply-accumulate) of a large-N FX correlator.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may include, link or call this file;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it. It shares no
 * code, header, table or constant with the CUDA library.
 *
 * What it computes (Sec. 1 and Sec. 2.5: the GPU layer performs the O(N^2) stage, multiplying every
 * pair of input spectra and integrating the products over groups of spectra; Table 1 note (a): the
 * four polarisation products of 256 dual-polarisation antennas; Sec. 2.6: the auto-correlation
 * (total power) cells):
 *
 *   for every channel f, every station pair (a, c) with a >= c and every polarisation pair (p, q):
 *       V_f[a p, c q] = sum_{t < T} x_{f, a p}(t) * conj(x_{f, c q}(t))          (exact int64)
 *   for every input m:
 *       A_f[m] = sum_{t < T} |x_{f, m}(t)|^2                                        (exact int64)
 *
 * Sample format (Sec. 2.2: requantisation of the F-engine output to 4+4 bits): one byte per complex
 * sample, high nibble = real part, low nibble = imaginary part, each a 4-bit two's-complement
 * integer in [-8, 7]. Input array layout uint8 in[T][C][N] (time slowest, input fastest: the data
 * after the corner turn of Sec. 2.3/2.4, grouped by channel). Input index n = n_pol * station + pol.
 *
 * Output layouts:
 *   cross[C][B_s][n_pol * n_pol][2]  int64 (re, im), B_s = S (S + 1) / 2, S = N / n_pol stations,
 *                                    pair index b(a, c) = a (a + 1) / 2 + c for a >= c,
 *                                    product index p * n_pol + q  (XX, XY, YX, YY for n_pol = 2)
 *   autos[C][N]                      int64
 *
 * The loops follow the definition directly: channel -> station pair -> polarisation pair -> time.
 * The only preprocessing is a per-channel gather of the samples into [input][time] order so that
 * the time loop walks memory contiguously; it does no arithmetic. Work may be split across
 * threads by channel only; every thread runs the same loop body.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* Sign-extend a 4-bit two's-complement nibble (Sec. 2.2: 4+4-bit complex samples). */
static int nibble_value(unsigned v) {
  v &= 0xFu;
  return (v & 0x8u) ? (int)v - 16 : (int)v;
}

static int real_part(uint8_t byte) { return nibble_value((unsigned)byte >> 4); }
static int imag_part(uint8_t byte) { return nibble_value((unsigned)byte); }

typedef struct {
  const uint8_t* in;
  int n_inputs, n_chans, n_time, n_pol;
  int64_t* cross;  /* may be NULL */
  int64_t* autos;  /* may be NULL */
  int chan_begin, chan_end;
  int status;
} job_t;

static void correlate_channel(const job_t* jb, int f, int8_t* re, int8_t* im) {
  const int N = jb->n_inputs, C = jb->n_chans, T = jb->n_time, np = jb->n_pol;
  const int S = N / np;
  const int64_t Bs = (int64_t)S * (S + 1) / 2;
  const int P = np * np;
  /* gather channel f into [input][time] */
  for (int t = 0; t < T; ++t) {
    const uint8_t* row = jb->in + ((size_t)t * C + f) * N;
    for (int n = 0; n < N; ++n) {
      re[(size_t)n * T + t] = (int8_t)real_part(row[n]);
      im[(size_t)n * T + t] = (int8_t)imag_part(row[n]);
    }
  }
  if (jb->cross) {
    for (int a = 0; a < S; ++a) {
      for (int c = 0; c <= a; ++c) {
        const int64_t b = (int64_t)a * (a + 1) / 2 + c;
        for (int p = 0; p < np; ++p) {
          for (int q = 0; q < np; ++q) {
            const int i = a * np + p, j = c * np + q;
            const int8_t* xr = re + (size_t)i * T;
            const int8_t* xi = im + (size_t)i * T;
            const int8_t* yr = re + (size_t)j * T;
            const int8_t* yi = im + (size_t)j * T;
            int64_t acc_re = 0, acc_im = 0;
            for (int t = 0; t < T; ++t) {
              /* x_i * conj(x_j) = (xr + i xi)(yr - i yi) */
              acc_re += (int64_t)xr[t] * yr[t] + (int64_t)xi[t] * yi[t];
              acc_im += (int64_t)xi[t] * yr[t] - (int64_t)xr[t] * yi[t];
            }
            int64_t* out = jb->cross + (((size_t)f * Bs + b) * P + (size_t)(p * np + q)) * 2;
            out[0] = acc_re;
            out[1] = acc_im;
          }
        }
      }
    }
  }
  if (jb->autos) {
    for (int m = 0; m < N; ++m) {
      const int8_t* xr = re + (size_t)m * T;
      const int8_t* xi = im + (size_t)m * T;
      int64_t acc = 0;
      for (int t = 0; t < T; ++t) acc += (int64_t)xr[t] * xr[t] + (int64_t)xi[t] * xi[t];
      jb->autos[(size_t)f * N + m] = acc;
    }
  }
}

static void* run_job(void* arg) {
  job_t* jb = (job_t*)arg;
  size_t n = (size_t)jb->n_inputs * (size_t)jb->n_time;
  int8_t* re = (int8_t*)malloc(n ? n : 1);
  int8_t* im = (int8_t*)malloc(n ? n : 1);
  if (!re || !im) {
    free(re);
    free(im);
    jb->status = -3;
    return NULL;
  }
  for (int f = jb->chan_begin; f < jb->chan_end; ++f) correlate_channel(jb, f, re, im);
  free(re);
  free(im);
  jb->status = 0;
  return NULL;
}

/*
 * Full correlation of every channel. Returns 0, -1 on bad arguments, -3 on allocation failure.
 * n_threads <= 1 runs on the calling thread.
 */
int oracle_correlate(const uint8_t* in, int n_inputs, int n_chans, int n_time, int n_pol,
                     int64_t* cross, int64_t* autos, int n_threads) {
  if (!in || n_inputs < 1 || n_chans < 1 || n_time < 0 || (n_pol != 1 && n_pol != 2) ||
      n_inputs % n_pol != 0)
    return -1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_chans) n_threads = n_chans;
  job_t* jobs = (job_t*)calloc((size_t)n_threads, sizeof(job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -3;
  }
  for (int k = 0; k < n_threads; ++k) {
    jobs[k].in = in;
    jobs[k].n_inputs = n_inputs;
    jobs[k].n_chans = n_chans;
    jobs[k].n_time = n_time;
    jobs[k].n_pol = n_pol;
    jobs[k].cross = cross;
    jobs[k].autos = autos;
    jobs[k].chan_begin = (int)((int64_t)n_chans * k / n_threads);
    jobs[k].chan_end = (int)((int64_t)n_chans * (k + 1) / n_threads);
    jobs[k].status = -1;
  }
  int rc = 0;
  if (n_threads == 1) {
    run_job(&jobs[0]);
    rc = jobs[0].status;
  } else {
    int started = 0;
    for (int k = 0; k < n_threads; ++k) {
      if (pthread_create(&th[k], NULL, run_job, &jobs[k]) != 0) break;
      ++started;
    }
    for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
    for (int k = started; k < n_threads; ++k) run_job(&jobs[k]);
    for (int k = 0; k < n_threads; ++k)
      if (jobs[k].status != 0) rc = jobs[k].status;
  }
  free(jobs);
  free(th);
  return rc;
}

/*
 * Individual visibility cells, for sampled checks of large runs: for each k,
 * out[2k], out[2k+1] = sum_t x_{f_k, i_k}(t) * conj(x_{f_k, j_k}(t)) with cells[3k..3k+2] = (f, i, j).
 * Any input indices i, j are accepted (not only the stored triangle). Returns 0 or -1.
 */
int oracle_cells(const uint8_t* in, int n_inputs, int n_chans, int n_time, int n_cells,
                 const int32_t* cells, int64_t* out) {
  if (!in || !cells || !out || n_inputs < 1 || n_chans < 1 || n_time < 0) return -1;
  for (int k = 0; k < n_cells; ++k) {
    const int f = cells[3 * k], i = cells[3 * k + 1], j = cells[3 * k + 2];
    if (f < 0 || f >= n_chans || i < 0 || i >= n_inputs || j < 0 || j >= n_inputs) return -1;
    int64_t acc_re = 0, acc_im = 0;
    for (int t = 0; t < n_time; ++t) {
      const uint8_t* row = in + ((size_t)t * n_chans + f) * n_inputs;
      const int xr = real_part(row[i]), xi = imag_part(row[i]);
      const int yr = real_part(row[j]), yi = imag_part(row[j]);
      acc_re += (int64_t)xr * yr + (int64_t)xi * yi;
      acc_im += (int64_t)xi * yr - (int64_t)xr * yi;
    }
    out[2 * k] = acc_re;
    out[2 * k + 1] = acc_im;
  }
  return 0;
}

/* Autocorrelations only (Sec. 2.6, total power), all channels. Returns 0 or -1. */
int oracle_autos(const uint8_t* in, int n_inputs, int n_chans, int n_time, int64_t* autos) {
  if (!in || !autos || n_inputs < 1 || n_chans < 1 || n_time < 0) return -1;
  for (int f = 0; f < n_chans; ++f)
    for (int m = 0; m < n_inputs; ++m) {
      int64_t acc = 0;
      for (int t = 0; t < n_time; ++t) {
        const uint8_t v = in[((size_t)t * n_chans + f) * n_inputs + m];
        const int xr = real_part(v), xi = imag_part(v);
        acc += (int64_t)xr * xr + (int64_t)xi * xi;
      }
      autos[(size_t)f * n_inputs + m] = acc;
    }
  return 0;
}
