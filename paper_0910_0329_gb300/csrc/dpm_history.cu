// dpm_history.cu -- one-history-per-thread transport (the paper's own layout,
// Sec. 2.2: each thread follows a source particle and all its secondaries
// with a private stack), the batch fold and the dose normalisation.
#include <cuda_runtime.h>

#include "dpm_device.cuh"
#include "dpm_kernels.h"

namespace dpm {

// Tally sink with run-length coalescing: consecutive deposits of one thread
// into the same voxel are summed in a register and issued as one 64-bit
// atomic add (exact, order-independent fixed point, 2^-32 MeV).  Real: the
// transport's arithmetic (float; double for the precision ablation).
template <class Real>
struct HistSinkT {
  static constexpr bool kSauter = true;  // DPM_SAUTER compiled in
  const RunParamsT<Real> &R;
  unsigned long long *slab = nullptr;
  int pend_v = -1;
  long long pend_q = 0;
  long long cnt[C_N];
  int err = 0;
  PartT<Real> *stack;
  int sp = 0, cap;

  __device__ HistSinkT(const RunParamsT<Real> &r, PartT<Real> *st, int c) : R(r), stack(st), cap(c) {
#pragma unroll
    for (int i = 0; i < C_N; ++i) cnt[i] = 0;
  }
  __device__ __forceinline__ static long long fx(Real e) { return Num<Real>::round_ll(e * Real(4294967296.0f)); }
  // energy counters (coarser quantum, see kCounterScale)
  __device__ __forceinline__ static long long fxc(Real e) { return Num<Real>::round_ll(e * Real(kCounterScaleF)); }
  __device__ __forceinline__ void flush() {
    if (pend_v >= 0 && pend_q != 0) {
      atomicAdd(slab + pend_v, (unsigned long long)pend_q);
      ++cnt[C_ATOM];
    }
    pend_v = -1;
    pend_q = 0;
  }
  __device__ __forceinline__ void deposit(int v, Real dE) {
    const long long q = fx(dE);
    if (v == pend_v) {
      pend_q += q;
    } else {
      flush();
      pend_v = v;
      pend_q = q;
    }
  }
  __device__ __forceinline__ void escape(Real E) { cnt[C_ESC] += fxc(E); }
  __device__ __forceinline__ void push(const PartT<Real> &q) {
    ++cnt[C_PUSH];
    if (sp < cap) {
      stack[sp++] = q;
    } else {
      err |= ERR_OVERFLOW;
      cnt[C_ESC] += fxc(q.E + (q.type == POSITRON ? Real(2) * Num<Real>::mc2 : Real(0)));
    }
  }
  __device__ __forceinline__ void error(int e) { err |= e; }
  __device__ __forceinline__ void count_step() { ++cnt[C_ESTEP]; }
  __device__ __forceinline__ void count_flight() { ++cnt[C_GFLIGHT]; }
  __device__ __forceinline__ void count_interaction() { ++cnt[C_GINT]; }
};
using HistSink = HistSinkT<float>;

template <class RP>
__device__ void reduce_counters(const long long *cnt, int err, const RP &R) {
#pragma unroll
  for (int i = 0; i < C_N; ++i) {
    long long v = cnt[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0) atomicAdd(R.counters + i, (unsigned long long)v);
  }
  int e = err;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e |= __shfl_down_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0 && e) atomicOr(R.err, e);
}

constexpr int kHistStack = 64;

// 8 resident blocks of 128 threads cap the registers at 64, as in the queue
// kernel: the extra spills cost less than the doubled occupancy gains
// (+26 % on 6 MV, +30 % on 20 MeV electrons against 128 registers).
template <class Real>
__global__ void __launch_bounds__(128, 8) k_history(const __grid_constant__ RunParamsT<Real> R, uint64_t batch_size) {
  PartT<Real> stack[kHistStack];
  HistSinkT<Real> s(R, stack, kHistStack);
  const size_t V = size_t(R.P.nx) * R.P.ny * R.P.nz;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t hl = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; hl < R.n; hl += stride) {
    s.slab = R.slabs + (hl / batch_size) * V;
    PartT<Real> p;
    const bool hit = make_primary(p, R, uint32_t(hl));
    s.cnt[C_EMIT] += HistSinkT<Real>::fxc(p.E);
    if (!hit) {
      s.cnt[C_MISS] += HistSinkT<Real>::fxc(p.E);
      continue;
    }
    s.sp = 0;
    s.stack[s.sp++] = p;
    while (s.sp > 0) {
      PartT<Real> q = s.stack[--s.sp];
      if (q.type == PHOTON) {
        int g = 0;
        while (photon_segment(q, R, s)) {
          if (++g >= kMaxPhotonSegments) {
            s.error(ERR_STEPCAP);
            s.deposit(vox(q, R.P), q.E);
            break;
          }
        }
      } else {
        int n = 0;
        while (electron_step(q, R, s)) {
          if (++n >= kMaxElectronSteps) {
            s.error(ERR_STEPCAP);
            s.deposit(vox(q, R.P), q.E);
            break;
          }
        }
      }
    }
    s.flush();
  }
  reduce_counters(s.cnt, s.err, R);
}

template <class Real>
static void launch_history_t(const RunParamsT<Real> &R, uint64_t batch_size, int sm_count, cudaStream_t st) {
  const int block = 128;  // the kernel's launch bound
  const uint64_t need = (R.n + block - 1) / block;
  const uint64_t cap = uint64_t(sm_count) * 16;
  const int grid = int(need < cap ? need : cap);
  cudaFuncSetAttribute(k_history<Real>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  k_history<Real><<<grid > 0 ? grid : 1, block, 0, st>>>(R, batch_size);
}

void launch_history(const RunParams &R, uint64_t batch_size, int sm_count, int block, cudaStream_t st) {
  (void)block;
  launch_history_t(R, batch_size, sm_count, st);
}

void launch_history_f64(const RunParamsT<double> &R, uint64_t batch_size, int sm_count, cudaStream_t st) {
  launch_history_t(R, batch_size, sm_count, st);
}

// ---------------------------------------------------------------------------
// The paper's own tally (Sec. 2.4), kept as an ablation of the exact one above.
// Each thread holds a sparse dose counter of kPaperCounter (voxel, energy)
// entries in its own memory: a deposit adds to its voxel's entry (searched
// from the newest, since consecutive deposits usually share a voxel) or opens
// a new one.  When the history ends, or the counter is full, the entries are
// added to a float dose array with atomic float additions.  kCas emulates the
// float addition with a compare-and-swap loop on the 32-bit word, the scheme
// the paper uses on a GPU without float atomics; otherwise the native float
// atomic add is used.  Float sums depend on the order of the additions, so
// this tally is not reproducible bit for bit; k_f32_to_fixed rounds it to
// the fixed-point slabs for the common fold.
// ---------------------------------------------------------------------------
constexpr int kPaperCounter = 128;
constexpr int kCasTries = 1 << 20;  // a bound on one CAS addition's retries

template <bool kCas>
__device__ __forceinline__ bool add_f32(float *a, float x) {
  if (!kCas) {
    atomicAdd(a, x);
    return true;
  }
  unsigned int *w = reinterpret_cast<unsigned int *>(a);
  unsigned int old = *w;
  for (int t = 0; t < kCasTries; ++t) {
    const unsigned int seen = old;
    old = atomicCAS(w, seen, __float_as_uint(__uint_as_float(seen) + x));
    if (old == seen) return true;
  }
  return false;
}

template <bool kCas>
struct PaperSink {
  static constexpr bool kSauter = false;
  const RunParams &R;
  float *fslab = nullptr;
  int n = 0;
  int lv[kPaperCounter];
  float le[kPaperCounter];
  long long cnt[C_N];
  int err = 0;
  Part *stack;
  int sp = 0, cap;

  __device__ PaperSink(const RunParams &r, Part *st, int c) : R(r), stack(st), cap(c) {
#pragma unroll
    for (int i = 0; i < C_N; ++i) cnt[i] = 0;
  }
  __device__ void flush() {
    for (int i = 0; i < n; ++i) {
      if (!add_f32<kCas>(fslab + lv[i], le[i])) err |= ERR_TIMEOUT;
    }
    cnt[C_ATOM] += n;
    n = 0;
  }
  __device__ void deposit(int v, float dE) {
    for (int i = n - 1; i >= 0; --i) {
      if (lv[i] == v) {
        le[i] += dE;
        return;
      }
    }
    if (n == kPaperCounter) flush();
    lv[n] = v;
    le[n] = dE;
    ++n;
  }
  // run counters exactly as HistSink keeps them, so that the energy balance
  // of both tallies is the same
  __device__ __forceinline__ void escape(float E) { cnt[C_ESC] += HistSink::fxc(E); }
  __device__ __forceinline__ void push(const Part &q) {
    ++cnt[C_PUSH];
    if (sp < cap) {
      stack[sp++] = q;
    } else {
      err |= ERR_OVERFLOW;
      cnt[C_ESC] += HistSink::fxc(q.E + (q.type == POSITRON ? 2.f * kMc2f : 0.f));
    }
  }
  __device__ __forceinline__ void error(int e) { err |= e; }
  __device__ __forceinline__ void count_step() { ++cnt[C_ESTEP]; }
  __device__ __forceinline__ void count_flight() { ++cnt[C_GFLIGHT]; }
  __device__ __forceinline__ void count_interaction() { ++cnt[C_GINT]; }
};

template <bool kCas>
__global__ void __launch_bounds__(128) k_history_paper(const __grid_constant__ RunParams R, uint64_t batch_size,
                                                       float *fslabs) {
  Part stack[kHistStack];
  PaperSink<kCas> s(R, stack, kHistStack);
  const size_t V = size_t(R.P.nx) * R.P.ny * R.P.nz;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t hl = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; hl < R.n; hl += stride) {
    s.fslab = fslabs + (hl / batch_size) * V;
    Part p;
    const bool hit = make_primary(p, R, uint32_t(hl));
    s.cnt[C_EMIT] += HistSink::fxc(p.E);
    if (!hit) {
      s.cnt[C_MISS] += HistSink::fxc(p.E);
      continue;
    }
    s.sp = 0;
    s.stack[s.sp++] = p;
    while (s.sp > 0) {
      Part q = s.stack[--s.sp];
      if (q.type == PHOTON) {
        int g = 0;
        while (photon_segment(q, R, s)) {
          if (++g >= kMaxPhotonSegments) {
            s.error(ERR_STEPCAP);
            s.deposit(vox(q, R.P), q.E);
            break;
          }
        }
      } else {
        int n = 0;
        while (electron_step(q, R, s)) {
          if (++n >= kMaxElectronSteps) {
            s.error(ERR_STEPCAP);
            s.deposit(vox(q, R.P), q.E);
            break;
          }
        }
      }
    }
    s.flush();
  }
  reduce_counters(s.cnt, s.err, R);
}

// Float dose slabs to the fixed-point slabs (nearest multiple of 2^-32 MeV).
__global__ void k_f32_to_fixed(const float *f, unsigned long long *slabs, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    slabs[i] = (unsigned long long)__double2ll_rn(double(f[i]) * 4294967296.0);
}

void launch_history_paper(const RunParams &R, uint64_t batch_size, bool cas, float *fslabs, size_t n_slab,
                          int sm_count, cudaStream_t st) {
  const int block = 128;
  const uint64_t need = (R.n + block - 1) / block;
  const uint64_t cap = uint64_t(sm_count) * 16;
  const int grid = int(need < cap ? need : cap);
  if (cas) {
    cudaFuncSetAttribute(k_history_paper<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    k_history_paper<true><<<grid > 0 ? grid : 1, block, 0, st>>>(R, batch_size, fslabs);
  } else {
    cudaFuncSetAttribute(k_history_paper<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    k_history_paper<false><<<grid > 0 ? grid : 1, block, 0, st>>>(R, batch_size, fslabs);
  }
  const size_t cgrid = (n_slab + 255) / 256 < size_t(sm_count) * 8 ? (n_slab + 255) / 256 : size_t(sm_count) * 8;
  k_f32_to_fixed<<<cgrid > 0 ? int(cgrid) : 1, 256, 0, st>>>(fslabs, R.slabs, n_slab);
}

// Sum the batch slabs of one run into S1 (exact int64) and Q = sum_b d_b^2/n_b.
__global__ void k_fold(const unsigned long long *slabs, int nb, size_t V, const double *inv_nb, long long *S1,
                       double *Q) {
  for (size_t v = size_t(blockIdx.x) * blockDim.x + threadIdx.x; v < V; v += size_t(gridDim.x) * blockDim.x) {
    long long s = 0;
    double q = 0.0;
    for (int b = 0; b < nb; ++b) {
      const long long d = (long long)slabs[size_t(b) * V + v];
      s += d;
      const double dd = double(d);
      q += dd * dd * inv_nb[b];
    }
    S1[v] += s;
    Q[v] += q;
  }
}

void launch_fold(const unsigned long long *slabs, int nb, size_t V, const double *inv_nb, long long *S1, double *Q,
                 int sm_count, cudaStream_t st) {
  const size_t need = (V + 255) / 256;
  const size_t cap = size_t(sm_count) * 8;
  const int grid = int(need < cap ? need : cap);
  k_fold<<<grid > 0 ? grid : 1, 256, 0, st>>>(slabs, nb, V, inv_nb, S1, Q);
}

// Dose (Gy per history) and its standard error from the batch statistics:
// per-history variance (Q - S1^2/n)/(B - 1), sigma of the mean sqrt(var/n).
__global__ void k_normalize(const long long *S1, const double *Q, const float *rho, size_t V, double n, double B,
                            double vox_cm3, double *dose, double *sigma) {
  for (size_t v = size_t(blockIdx.x) * blockDim.x + threadIdx.x; v < V; v += size_t(gridDim.x) * blockDim.x) {
    const double s1 = double(S1[v]);
    const double conv = kMeVtoJ / (double(rho[v]) * vox_cm3 * 1e-3) / kTallyScale;
    if (dose) dose[v] = n > 0 ? s1 / n * conv : 0.0;
    if (sigma) {
      double var = 0.0;
      if (B > 1.0 && n > 0) var = fmax(Q[v] - s1 * s1 / n, 0.0) / (B - 1.0);
      sigma[v] = n > 0 ? sqrt(var / n) * conv : 0.0;
    }
  }
}

void launch_normalize(const long long *S1, const double *Q, const float *rho, size_t V, double n, double B,
                      double vox_cm3, double *dose, double *sigma, int sm_count, cudaStream_t st) {
  const size_t need = (V + 255) / 256;
  const size_t cap = size_t(sm_count) * 8;
  const int grid = int(need < cap ? need : cap);
  k_normalize<<<grid > 0 ? grid : 1, 256, 0, st>>>(S1, Q, rho, V, n, B, vox_cm3, dose, sigma);
}

// D_max search for the stop rule: a 64-bit key (dose as float bits, which
// order like the values for non-negative doses, above the voxel index) reduced
// with atomicMax; then one thread evaluates dose and sigma at the winner.
__global__ void k_dmax_key(const long long *S1, const float *rho, size_t V, double vox_cm3,
                           unsigned long long *key) {
  unsigned long long best = 0;
  for (size_t v = size_t(blockIdx.x) * blockDim.x + threadIdx.x; v < V; v += size_t(gridDim.x) * blockDim.x) {
    const double s1 = double(S1[v]);
    if (s1 <= 0) continue;
    const float dose = float(s1 * kMeVtoJ / (double(rho[v]) * vox_cm3 * 1e-3));
    const unsigned long long k = (uint64_t(__float_as_uint(dose)) << 32) | uint64_t(uint32_t(v));
    best = k > best ? k : best;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, best, o);
    best = other > best ? other : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(key, best);
}

__global__ void k_dmax_eval(const long long *S1, const double *Q, const float *rho, double n, double B,
                            double vox_cm3, const unsigned long long *key, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  out[0] = out[1] = 0.0;
  out[2] = -1.0;
  if (*key == 0 || n <= 0) return;
  const size_t v = size_t(uint32_t(*key));
  const double s1 = double(S1[v]);
  const double conv = kMeVtoJ / (double(rho[v]) * vox_cm3 * 1e-3) / kTallyScale;
  const double var = B > 1.0 ? fmax(Q[v] - s1 * s1 / n, 0.0) / (B - 1.0) : 0.0;
  out[0] = s1 / n * conv;
  out[1] = sqrt(var / n) * conv;
  out[2] = double(v);
}

void launch_dmax(const long long *S1, const double *Q, const float *rho, size_t V, double n, double B, double vox_cm3,
                 unsigned long long *key, double *out, int sm_count, cudaStream_t st) {
  cudaMemsetAsync(key, 0, sizeof(unsigned long long), st);
  const size_t need = (V + 255) / 256;
  const size_t cap = size_t(sm_count) * 8;
  const int grid = int(need < cap ? need : cap);
  k_dmax_key<<<grid > 0 ? grid : 1, 256, 0, st>>>(S1, rho, V, vox_cm3, key);
  k_dmax_eval<<<1, 32, 0, st>>>(S1, Q, rho, n, B, vox_cm3, key, out);
}

}  // namespace dpm
