// dpm_device.cuh -- device-side transport physics, shared by the transport
// kernels: FP32 (the product path) and FP64 (the precision ablation) are two
// instantiations of the same templates on the real type.  Every function follows the DPM scheme of Sec. 2.1 with
// the closed-form model tabulated by dpm_tables.cpp.
//
// A "context" C supplies what a particle's history needs: C.T (tables), C.P
// (phantom), C.S (source), C.first, C.key0, C.key1 (history numbering and
// Philox key).  RunParams (one run) and JobCtx (one entry of a batch) both
// provide these members.
//
// A "sink" object receives what the physics produces:
//   sink.deposit(v, dE)  energy dE (MeV) deposited in voxel v
//   sink.escape(E)       energy carried out of the phantom
//   sink.push(part)      a secondary particle to be transported later
//   sink.error(bits)     a bounded loop gave up
// and says which optional physics its kernel compiles in:
//   Sink::kSauter        photoelectron angles (DPM_SAUTER)
#pragma once

#include <cuda_runtime.h>

#include "dpm_internal.h"

namespace dpm {

constexpr float kMc2f = 0.51099895f;
constexpr int kMaxElectronSteps = 200000;  // per particle; far above any real track
constexpr int kMaxPhotonFlights = 100000;
constexpr int kMaxPhotonSegments = 10000;  // Compton scatters of one photon

// Rarely executed physics (source, interactions, hard events, annihilation)
// is inlined: measured on GB300, calls to out-of-line copies cost more than
// the instruction-cache pressure they save.  DPM_COLD_NOINLINE keeps it out
// of line (for measurements).
#ifdef DPM_COLD_NOINLINE
#define DPM_COLD __noinline__
#else
#define DPM_COLD __forceinline__
#endif

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): counter-based, so a particle's random
// numbers depend only on its identity, never on the thread that runs it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// ---------------------------------------------------------------------------
// Arithmetic of one precision.  The transport is FP32 (Sec. 2.3), with the
// hardware approximations where their error is far below the tables' and the
// statistics' (each use is argued where it is made); the FP64 instantiation
// of the same code takes the correctly rounded double functions throughout
// and serves to measure what single precision costs.
// ---------------------------------------------------------------------------
template <class Real>
struct Num;

template <>
struct Num<float> {
  static constexpr float mc2 = 0.51099895f;
  static constexpr float inf = 3.0e38f;
  static __device__ __forceinline__ float log_hw(float x) { return __logf(x); }
  static __device__ __forceinline__ float log2_hw(float x) { return __log2f(x); }
  static __device__ __forceinline__ float exp_hw(float x) { return __expf(x); }
  static __device__ __forceinline__ float div_hw(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
  // sine and cosine of pi*t for t in [-1, 1)
  static __device__ __forceinline__ void sincospi_hw(float t, float *s, float *c) { __sincosf(3.14159265f * t, s, c); }
  static __device__ __forceinline__ void sincospi(float t, float *s, float *c) { sincospif(t, s, c); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ float min(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float max(float a, float b) { return fmaxf(a, b); }
  static __device__ __forceinline__ float floor(float x) { return floorf(x); }
  static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float log(float x) { return logf(x); }
  static __device__ __forceinline__ float exp(float x) { return expf(x); }
  static __device__ __forceinline__ float log1p(float x) { return log1pf(x); }
  static __device__ __forceinline__ float acos(float x) { return acosf(x); }
  static __device__ __forceinline__ float cos(float x) { return cosf(x); }
  static __device__ __forceinline__ long long round_ll(float x) { return __float2ll_rn(x); }
  // uniform on (0, 1] from the top 24 bits: (k + 1/2) 2^-24 for k = x >> 8,
  // in one rounding (the top values round to 1)
  static __device__ __forceinline__ float u01(uint32_t x) {
    return fmaf(float(x >> 8), 1.0f / 16777216.0f, 1.0f / 33554432.0f);
  }
  static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ float4 ld4(const float4 *p) { return __ldg(p); }
};

template <>
struct Num<double> {
  static constexpr double mc2 = 0.51099895;
  static constexpr double inf = 1.0e300;
  static __device__ __forceinline__ double log_hw(double x) { return ::log(x); }
  static __device__ __forceinline__ double log2_hw(double x) { return ::log2(x); }
  static __device__ __forceinline__ double exp_hw(double x) { return ::exp(x); }
  static __device__ __forceinline__ double div_hw(double a, double b) { return a / b; }
  static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
  static __device__ __forceinline__ void sincospi_hw(double t, double *s, double *c) { ::sincospi(t, s, c); }
  static __device__ __forceinline__ void sincospi(double t, double *s, double *c) { ::sincospi(t, s, c); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ double min(double a, double b) { return ::fmin(a, b); }
  static __device__ __forceinline__ double max(double a, double b) { return ::fmax(a, b); }
  static __device__ __forceinline__ double floor(double x) { return ::floor(x); }
  static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  static __device__ __forceinline__ double log(double x) { return ::log(x); }
  static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
  static __device__ __forceinline__ double log1p(double x) { return ::log1p(x); }
  static __device__ __forceinline__ double acos(double x) { return ::acos(x); }
  static __device__ __forceinline__ double cos(double x) { return ::cos(x); }
  static __device__ __forceinline__ long long round_ll(double x) { return __double2ll_rn(x); }
  // the same deviate as the FP32 path's, (k + 1/2) 2^-24, exactly
  static __device__ __forceinline__ double u01(uint32_t x) { return (double(x >> 8) + 0.5) * (1.0 / 16777216.0); }
  static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
  static __device__ __forceinline__ Dbl4 ld4(const Dbl4 *p) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return Dbl4{a.x, a.y, b.x, b.y};
  }
};

__device__ __forceinline__ float u01(uint32_t x) { return Num<float>::u01(x); }

// -ln(u) for an exponential free path, with the hardware logarithm (absolute
// error about 2^-21 near u = 1, far below the paths' statistical spread); the
// clamp keeps a rounding just above zero from reversing a flight.
template <class Real>
__device__ __forceinline__ Real neglog(Real u) {
  return Num<Real>::max(-Num<Real>::log_hw(u), Real(0));
}

// ---------------------------------------------------------------------------
// Particle state.  (ix, iy, iz) are tracked exactly across voxel faces.
// ---------------------------------------------------------------------------
enum : int { PHOTON = 0, ELECTRON = 1, POSITRON = 2 };

template <class Real>
struct PartT {
  Real x, y, z, u, v, w, E;
  int ix, iy, iz;
  uint32_t id_lo, id_hi;  // particle id within its history
  uint32_t ctr;           // next Philox block of this particle
  uint32_t hist;          // history index relative to the run (or job)
  int type;
  int job;                // index in the batch's job table (0 for a single run)
};
using Part = PartT<float>;

// Philox key of a history: seed hash xor the global history id; the third
// counter word carries more seed bits so that different seeds never share
// streams.
template <class Real, class Ctx>
__device__ __forceinline__ uint4 draw(PartT<Real> &p, const Ctx &R) {
  const uint64_t h = R.first + p.hist;
  const uint4 c = make_uint4(p.ctr++, p.id_lo, p.id_hi, R.key0 ^ 0x5bd1e995u);
  return philox4x32_10(c, R.key0 ^ uint32_t(h), R.key1 ^ uint32_t(h >> 32));
}

// Context of one batch job: references into the job table (global memory)
// plus the history numbering held in registers.
struct JobCtx {
  const DevTables &T;
  const DevPhantom &P;
  const DevSource &S;
  uint64_t first;
  uint32_t key0, key1;
};

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// A secondary of p: same position and voxel, fresh random stream whose id is
// a hash of the parent's id, the parent's draw counter and an ordinal.
template <class Real>
__device__ __forceinline__ PartT<Real> child(const PartT<Real> &p, int type, uint32_t ordinal) {
  PartT<Real> c = p;
  c.type = type;
  c.ctr = 0;
  const uint64_t pid = (uint64_t(p.id_hi) << 32) | p.id_lo;
  const uint64_t id = mix64(pid * 0x9E3779B97F4A7C15ull + ((uint64_t(p.ctr) << 8) | ordinal) + 0x632BE59BD9B4E019ull);
  c.id_lo = uint32_t(id);
  c.id_hi = uint32_t(id >> 32);
  return c;
}

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
template <class Real>
__device__ __forceinline__ int vox(const PartT<Real> &p, const DevPhantomT<Real> &P) {
  return p.ix + P.nx * (p.iy + P.ny * p.iz);
}

// Path length to the next face along one axis.  The hardware division (2 ulp)
// suffices: a step that reaches a face puts the coordinate on the face
// exactly (cross_face), so its error only moves the step length by 2 ulp.
template <class Real>
__device__ __forceinline__ Real face_dist(Real x, Real u, int i, Real d) {
  using N = Num<Real>;
  if (u > Real(0)) return N::max(N::div_hw(N::fma(Real(i + 1), d, -x), u), Real(0));
  if (u < Real(0)) return N::max(N::div_hw(N::fma(Real(i), d, -x), u), Real(0));
  return N::inf;
}

template <class Real>
__device__ __forceinline__ Real dist_to_face(const PartT<Real> &p, const DevPhantomT<Real> &P, int &axis) {
  Real t = face_dist(p.x, p.u, p.ix, P.dx);
  axis = 0;
  const Real ty = face_dist(p.y, p.v, p.iy, P.dy);
  if (ty < t) { t = ty; axis = 1; }
  const Real tz = face_dist(p.z, p.w, p.iz, P.dz);
  if (tz < t) { t = tz; axis = 2; }
  return t;
}

template <class Real>
__device__ __forceinline__ void move(PartT<Real> &p, Real s) {
  using N = Num<Real>;
  p.x = N::fma(s, p.u, p.x);
  p.y = N::fma(s, p.v, p.y);
  p.z = N::fma(s, p.w, p.z);
}

// Step into the neighbour across `axis`; false if that leaves the phantom.
template <class Real>
__device__ __forceinline__ bool cross_face(PartT<Real> &p, const DevPhantomT<Real> &P, int axis) {
  if (axis == 0) {
    if (p.u > Real(0)) { p.ix += 1; p.x = Real(p.ix) * P.dx; } else { p.x = Real(p.ix) * P.dx; p.ix -= 1; }
    return p.ix >= 0 && p.ix < P.nx;
  }
  if (axis == 1) {
    if (p.v > Real(0)) { p.iy += 1; p.y = Real(p.iy) * P.dy; } else { p.y = Real(p.iy) * P.dy; p.iy -= 1; }
    return p.iy >= 0 && p.iy < P.ny;
  }
  if (p.w > Real(0)) { p.iz += 1; p.z = Real(p.iz) * P.dz; } else { p.z = Real(p.iz) * P.dz; p.iz -= 1; }
  return p.iz >= 0 && p.iz < P.nz;
}

// Voxel containing a point known to be inside the phantom.
template <class Real>
__device__ __forceinline__ void locate(PartT<Real> &p, const DevPhantomT<Real> &P) {
  using N = Num<Real>;
  p.ix = min(max(int(N::floor(p.x / P.dx)), 0), P.nx - 1);
  p.iy = min(max(int(N::floor(p.y / P.dy)), 0), P.ny - 1);
  p.iz = min(max(int(N::floor(p.z / P.dz)), 0), P.nz - 1);
}

// Rotate the direction by polar cosine c and azimuth pi*h (h in half turns).
// h is reduced modulo 2 to [-1, 1), where the hardware sine and cosine are
// accurate to about 2^-21 absolute; the direction is renormalised below.
template <class Real>
__device__ __forceinline__ void rotate(Real &u, Real &v, Real &w, Real c, Real h) {
  using N = Num<Real>;
  c = N::min(N::max(c, Real(-1)), Real(1));
  const Real c2 = N::max(Real(0), N::fma(-c, c, Real(1)));
  const Real s = c2 * N::rsqrt(N::max(c2, Real(1e-30f)));  // sin(theta) by the hardware 1/sqrt
  Real sp, cp;
  const Real t = h - Real(2) * N::floor(Real(0.5) * h + Real(0.5));  // h modulo 2, in [-1, 1)
  N::sincospi_hw(t, &sp, &cp);
  const Real r2 = N::fma(u, u, v * v);
  Real nu, nv, nw;
  if (r2 < Real(1e-10f)) {
    nu = s * cp;
    nv = s * sp;
    nw = (w >= Real(0)) ? c : -c;
  } else {
    const Real ir = N::rsqrt(r2), r = r2 * ir, a = s * ir;  // hardware 1/sqrt; renormalised below
    nu = N::fma(u, c, a * N::fma(u * w, cp, -(v * sp)));
    nv = N::fma(v, c, a * N::fma(v * w, cp, u * sp));
    nw = N::fma(w, c, -(s * r) * cp);
  }
  const Real n = N::rsqrt(N::fma(nu, nu, N::fma(nv, nv, nw * nw)));
  u = nu * n;
  v = nv * n;
  w = nw * n;
}

// ---------------------------------------------------------------------------
// Table access: linear interpolation on a uniform ln(E) grid
// ---------------------------------------------------------------------------
template <class Real>
struct EIdxT {
  int i;
  Real f;
};
using EIdx = EIdxT<float>;

// Grid position x (fractional node index) clamped to the table.
template <class Real>
__device__ __forceinline__ EIdxT<Real> eidx_x(const DevTablesT<Real> &T, Real x) {
  using N = Num<Real>;
  x = N::min(N::max(x, Real(0)), Real(T.n_e - 1) - Real(1e-3f));
  EIdxT<Real> e;
  e.i = int(x);
  e.f = x - Real(e.i);
  return e;
}

// Fractional node index of energy E on the uniform ln E grid, from the
// hardware base-2 logarithm in one FMA (x_lg2 = ln 2 / spacing, x_lo = -ln E_lo
// / spacing).  The intrinsic's documented error (2 ulp of log2 E, within
// 7e-7 of ln E on the tables' range) moves the position by at most 2.5e-4 of
// a node spacing at 2048 nodes: an interpolation error well below the
// tables' own.
template <class Real>
__device__ __forceinline__ Real egrid(const DevTablesT<Real> &T, Real E) {
  return Num<Real>::fma(Num<Real>::log2_hw(E), T.x_lg2, T.x_lo);
}

template <class Real>
__device__ __forceinline__ EIdxT<Real> eidx(const DevTablesT<Real> &T, Real E) {
  return eidx_x(T, egrid(T, E));
}

template <class Real>
__device__ __forceinline__ Real lerp(Real a, Real b, Real f) {
  return Num<Real>::fma(f, b - a, a);
}

// The per-material tables hold, for every node, its four values and their
// differences to the next node (a 32-byte record in FP32): one interpolation
// reads one aligned sector and takes one FMA per component, with the same
// result as interpolating between the two nodes (the difference is the same
// subtraction, done when the table is uploaded).
template <class V4, class Real>
__device__ __forceinline__ V4 lerp_node(const V4 *b, Real f) {
  using N = Num<Real>;
  const V4 v = N::ld4(b), d = N::ld4(b + 1);
  V4 o;
  o.x = N::fma(f, d.x, v.x);
  o.y = N::fma(f, d.y, v.y);
  o.z = N::fma(f, d.z, v.z);
  o.w = N::fma(f, d.w, v.w);
  return o;
}

template <class V4, class Real>
__device__ __forceinline__ Real lerp_node_x(const V4 *b, Real f) {
  return Num<Real>::fma(f, Num<Real>::ld(&b[1].x), Num<Real>::ld(&b[0].x));
}

template <class Real>
__device__ __forceinline__ typename Vec4<Real>::type el_at(const DevTablesT<Real> &T, int m, EIdxT<Real> e) {
  return lerp_node(T.el + 2 * (size_t(m) * T.n_e + e.i), e.f);
}

template <class Real>
__device__ __forceinline__ Real el_range(const DevTablesT<Real> &T, int m, EIdxT<Real> e) {
  return lerp_node_x(T.el + 2 * (size_t(m) * T.n_e + e.i), e.f);
}

template <class Real>
__device__ __forceinline__ typename Vec4<Real>::type ph_at(const DevTablesT<Real> &T, int m, EIdxT<Real> e) {
  return lerp_node(T.ph + 2 * (size_t(m) * T.n_e + e.i), e.f);
}

template <class Real>
__device__ __forceinline__ Real ph_mu(const DevTablesT<Real> &T, int m, EIdxT<Real> e) {
  return lerp_node_x(T.ph + 2 * (size_t(m) * T.n_e + e.i), e.f);
}

template <class Real>
__device__ __forceinline__ Real samp(const SampTabT<Real> &t, Real lnE, Real u) {
  using N = Num<Real>;
  Real x = (lnE - t.lnE0) * t.inv_dlnE;
  x = N::min(N::max(x, Real(0)), Real(t.ne - 1) - Real(1e-3f));
  const int i = int(x);
  const Real fx = x - Real(i);
  const Real yk = u * Real(t.nu - 1);
  const int k = min(int(yk), t.nu - 2);
  const Real fy = yk - Real(k);
  const Real *r0 = t.y + size_t(i) * t.nu + k;
  const Real a = lerp(N::ld(r0), N::ld(r0 + 1), fy);
  const Real b = lerp(N::ld(r0 + t.nu), N::ld(r0 + t.nu + 1), fy);
  return lerp(a, b, fx);
}

// A of the random-hinge distribution for a step of x = s/lambda1: the table is
// ln A against logit(q), q = 1 - exp(-x); beyond its ends ln A grows like logit(q).
template <class Real>
__device__ __forceinline__ Real msc_A(const DevTablesT<Real> &T, Real x) {
  using N = Num<Real>;
  // q = 1 - exp(-x): a Taylor polynomial below x = 0.1 (truncation under
  // 1e-7 relative), the hardware exponential above (2 ulp of exp(-x), at
  // most 3e-6 of q); the hardware logarithm then moves the table position
  // by a few 1e-6.  (FP64: 1 - exp(-x) without cancellation by expm1.)
  Real q;
  if (sizeof(Real) == 4)
    q = x < Real(0.1f) ? x * N::fma(-x, N::fma(-x, N::fma(-x, Real(1.f / 24.f), Real(1.f / 6.f)), Real(0.5f)), Real(1))
                       : Real(1) - N::exp_hw(-x);
  else
    q = -::expm1(double(-x));
  const Real lg = N::log_hw(q) + x;
  const Real t = (lg - T.msc_x0) * T.msc_inv_dx;
  Real lA;
  if (!(t > Real(0))) {  // also catches NaN
    lA = N::ld(T.msc_lnA) + (lg - T.msc_x0);
  } else if (t >= Real(T.msc_n - 1)) {
    lA = N::ld(T.msc_lnA + T.msc_n - 1) + (lg - (T.msc_x0 + Real(T.msc_n - 1) / T.msc_inv_dx));
  } else {
    const int i = int(t);
    lA = lerp(N::ld(T.msc_lnA + i), N::ld(T.msc_lnA + i + 1), t - Real(i));
  }
  return N::exp_hw(N::min(lA, Real(60)));  // hardware exponential: a few ulp at the ln A of real steps
}

// 1 - mu of the hinge distribution by its inverse CDF (hardware division,
// 2 ulp: far below the table's interpolation error).
template <class Real>
__device__ __forceinline__ Real msc_sample(Real A, Real xi) {
  return Num<Real>::div_hw(Real(2) * A * xi, Real(1) + A - xi);
}

// Kinetic energy after a CSDA mass path mp from T0 (range R0, stopping power S0
// at T0): Euler estimate refined by one Newton step on the range table.  For
// a step losing at most 5 % of T the Euler error is about (dT)^2 |S'|/(2S);
// the Newton step squares it, to about 1e-4 of the step's loss at 0.2 MeV
// and far less above.  A second step (one more dependent table load on the
// electron's critical path) measured 2-4 % slower.
template <class Real>
__device__ __forceinline__ Real csda_energy(const DevTablesT<Real> &T, int m, Real T0, Real R0, Real S0, Real mp) {
  using N = Num<Real>;
  const Real Rt = R0 - mp;
  const Real T1 = N::max(N::fma(-mp, S0, T0), Real(0.5) * T0);
  const typename Vec4<Real>::type r = el_at(T, m, eidx(T, T1));
  return N::min(N::fma(-(r.x - Rt), r.y, T1), T0);
}

// Synthetic 6 MV spectrum f(E) ~ (1 - E/6) E^-1/2 on [0.25, 6] MeV: the CDF in
// t = sqrt(E) is the cubic 2t - t^3/9; its middle root by the trigonometric
// formula.  The constants are given to the precision of the type.
template <class Real>
__device__ __forceinline__ Real spectrum_6mv(Real u) {
  using N = Num<Real>;
  const bool f32 = sizeof(Real) == 4;
  const Real F0 = f32 ? Real(0.98611111f) : Real(0.98611111111111111);  // 2(0.5) - 0.5^3/9
  const Real F1 = f32 ? Real(3.26598632f) : Real(3.2659863237109041);   // 2 sqrt6 - 6 sqrt6/9
  const Real c = F0 + u * (F1 - F0);
  const Real k3 = f32 ? Real(-0.30618622f) : Real(-0.30618621784789726);  // -(3/4) / sqrt(6)
  const Real arg = N::min(N::max(k3 * c, Real(-1)), Real(1));
  const Real s6 = f32 ? Real(4.89897949f) : Real(4.8989794855663562);   // 2 sqrt6
  const Real third = f32 ? Real(1.f / 3.f) : Real(1.0 / 3.0);
  const Real tpi3 = f32 ? Real(2.09439510f) : Real(2.0943951023931955);  // 2 pi / 3
  const Real t = s6 * N::cos(N::acos(arg) * third - tpi3);
  return N::min(N::max(t * t, Real(0.25)), Real(6));
}

// Photoelectron polar angle (an option, DPM_SAUTER): Sauter's K-shell
// distribution sin^2(th)/(1 - b cos th)^4 [1 + g(g-1)(g-2)(1 - b cos th)/2]
// (b, g the electron's speed and Lorentz factor).  In x = nu/(A+nu), with
// nu = 1 - cos th and A = 1/b - 1, its density is x(2 - (2+A)x)(1 + AB/(1-x))
// on [0, 2/(2+A)], B = b g(g-1)(g-2)/2; the table holds x / x_max on a ln T
// grid against w = acos(1 - 2u)/pi of the uniform deviate u, in which both
// ends of the inverse CDF are linear (dpm_tables.cpp).  Returns nu.
template <class Real>
__device__ __forceinline__ Real sauter_nu(const DevTablesT<Real> &T, Real E, Real lnE, Real u) {
  using N = Num<Real>;
  const Real A = (E + N::mc2) / N::sqrt(E * (E + Real(2) * N::mc2)) - Real(1);
  const Real w = N::acos(Real(1) - Real(2) * u) * Real(0.318309886183790672);  // 1/pi
  const Real x = samp(T.sauter, lnE, w) * (Real(2) / (Real(2) + A));
  return A * x / (Real(1) - x);
}

// ---------------------------------------------------------------------------
// Emission helpers: below the absorption energy a new particle deposits on the
// spot (Sec. 3); a positron then also annihilates.
// ---------------------------------------------------------------------------
template <class Real, class Ctx, class Sink>
__device__ DPM_COLD void annihilate(PartT<Real> &p, const Ctx &R, Sink &s) {
  using N = Num<Real>;
  const uint4 r = draw(p, R);
  const Real cz = Real(2) * N::u01(r.x) - Real(1);
  const Real sz = N::sqrt(N::max(Real(0), Real(1) - cz * cz));
  Real sp, cp;
  N::sincospi(Real(2) * N::u01(r.y), &sp, &cp);
  PartT<Real> g = child(p, PHOTON, 1);
  g.E = N::mc2;
  g.u = sz * cp;
  g.v = sz * sp;
  g.w = cz;
  s.push(g);
  PartT<Real> h = child(p, PHOTON, 2);
  h.E = N::mc2;
  h.u = -g.u;
  h.v = -g.v;
  h.w = -g.w;
  s.push(h);
}

template <class Real, class Ctx, class Sink>
__device__ void emit_charged(PartT<Real> &q, const Ctx &R, Sink &s) {
  if (q.E > R.T.eabs_e) {
    s.push(q);
    return;
  }
  s.deposit(vox(q, R.P), q.E);
  if (q.type == POSITRON) annihilate(q, R, s);
}

template <class Real, class Ctx, class Sink>
__device__ void emit_photon(PartT<Real> &q, const Ctx &R, Sink &s) {
  if (q.E > R.T.eabs_g) s.push(q);
  else s.deposit(vox(q, R.P), q.E);
}

template <class Real, class Ctx, class Sink>
__device__ void absorb_charged(PartT<Real> &p, const Ctx &R, Sink &s) {
  s.deposit(vox(p, R.P), p.E);
  if (p.type == POSITRON) annihilate(p, R, s);
}

// ---------------------------------------------------------------------------
// Source (Sec. 3): point source at SAD from the isocentre, uniform over the
// field rectangle in the isocentre plane, flown to the phantom surface.
// Returns false if the ray misses the phantom.
// ---------------------------------------------------------------------------
template <class Real, class Ctx>
__device__ DPM_COLD bool make_primary(PartT<Real> &p, const Ctx &R, uint32_t hl) {
  using N = Num<Real>;
  const auto &S = R.S;
  const auto &P = R.P;
  p.hist = hl;
  p.job = 0;
  p.id_lo = 1u;
  p.id_hi = 0u;
  p.ctr = 0;
  p.type = (S.particle == 0) ? PHOTON : ELECTRON;
  const uint4 r = draw(p, R);
  const Real a = (N::u01(r.x) - Real(0.5)) * S.fx, b = (N::u01(r.y) - Real(0.5)) * S.fy;
  Real dx = S.cx + a * S.e1x - S.sx, dy = S.cy + b - S.sy, dz = S.cz + a * S.e1z - S.sz;
  const Real n = N::rsqrt(dx * dx + dy * dy + dz * dz);
  dx *= n;
  dy *= n;
  dz *= n;
  p.E = (S.spectrum == 1) ? spectrum_6mv(N::u01(r.z)) : S.energy;
  const Real L[3] = {P.nx * P.dx, P.ny * P.dy, P.nz * P.dz};
  const Real o[3] = {S.sx, S.sy, S.sz}, d[3] = {dx, dy, dz};
  Real t0 = Real(0), t1 = N::inf;
  int face = -1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (d[k] == Real(0)) {
      if (o[k] < Real(0) || o[k] > L[k]) return false;
      continue;
    }
    Real ta = (Real(0) - o[k]) / d[k], tb = (L[k] - o[k]) / d[k];
    if (ta > tb) { const Real t = ta; ta = tb; tb = t; }
    if (ta > t0) { t0 = ta; face = k; }
    t1 = N::min(t1, tb);
  }
  if (!(t1 > t0)) return false;
  p.x = N::fma(t0, dx, S.sx);
  p.y = N::fma(t0, dy, S.sy);
  p.z = N::fma(t0, dz, S.sz);
  p.u = dx;
  p.v = dy;
  p.w = dz;
  if (face == 0) p.x = dx > Real(0) ? Real(0) : L[0];
  if (face == 1) p.y = dy > Real(0) ? Real(0) : L[1];
  if (face == 2) p.z = dz > Real(0) ? Real(0) : L[2];
  locate(p, P);
  return true;
}

// ---------------------------------------------------------------------------
// Photons (Sec. 2.1): Woodcock flights over the majorant, then an interaction.
// Returns true while the photon is alive (after a Compton scatter).
// ---------------------------------------------------------------------------
template <class Real, class Ctx, class Sink>
__device__ DPM_COLD bool photon_interact(PartT<Real> &p, const Ctx &R, Sink &s, EIdxT<Real> e, int m) {
  using N = Num<Real>;
  const auto &T = R.T;
  const uint4 r = draw(p, R);
  const typename Vec4<Real>::type c = ph_at(T, m, e);
  const Real u0 = N::u01(r.x);
  const Real E = p.E, k = E / N::mc2, lnE = N::log(E);
  bool pair = u0 >= c.y + c.z;
  Real lo = Real(0), hi = Real(0);
  if (pair) {
    const Real two_sqrt_e = sizeof(Real) == 4 ? Real(3.29744254f) : Real(3.2974425414002564);  // 2 e^{1/2}
    const Real disc = Real(1) - two_sqrt_e / k;
    if (k <= Real(2) || disc <= Real(0)) {
      pair = false;  // below the model's threshold (interpolation edge): scatter instead
    } else {
      const Real sq = N::sqrt(disc);
      lo = N::max(Real(1) / k, Real(0.5) * (Real(1) - sq));
      hi = N::min(Real(1) - Real(1) / k, Real(0.5) * (Real(1) + sq));
      if (!(hi > lo)) pair = false;
    }
  }
  if (!pair && u0 >= c.y && u0 < c.y + c.z) {
    // photoelectric absorption: the electron takes the photon energy and
    // direction, or (DPM_SAUTER, in the kernels whose sink compiles it in)
    // leaves at Sauter's polar angle about it
    PartT<Real> el = child(p, ELECTRON, 1);
    if constexpr (Sink::kSauter) {
      if ((T.flags & DPM_SAUTER) && E > T.eabs_e)
        rotate(el.u, el.v, el.w, Real(1) - sauter_nu(T, E, lnE, N::u01(r.y)), Real(2) * N::u01(r.z));
    }
    emit_charged(el, R, s);
    return false;
  }
  if (pair) {
    const Real eps = lo + samp(T.pair, lnE, N::u01(r.y)) * (hi - lo);
    PartT<Real> a = child(p, ELECTRON, 1), b = child(p, POSITRON, 2);
    a.E = N::max(eps * E - N::mc2, Real(0));
    b.E = N::max((Real(1) - eps) * E - N::mc2, Real(0));
    emit_charged(a, R, s);
    emit_charged(b, R, s);
    return false;
  }
  // Compton (Klein-Nishina): y = ln(eps)/ln(eps0)
  const Real l0 = -N::log1p(Real(2) * k);
  const Real eps = N::exp(samp(T.kn, lnE, N::u01(r.y)) * l0);
  const Real Ep = eps * E, Te = E - Ep;
  const Real cth = Real(1) - (Real(1) / eps - Real(1)) / k;
  const Real h = Real(2) * N::u01(r.z);  // azimuth in half turns
  PartT<Real> el = child(p, ELECTRON, 1);
  el.E = Te;
  const Real pe = N::sqrt(Te * (Te + Real(2) * N::mc2));
  const Real ce = pe > Real(0) ? (E - Ep * cth) / pe : Real(1);
  rotate(el.u, el.v, el.w, ce, h + Real(1));
  emit_charged(el, R, s);
  rotate(p.u, p.v, p.w, cth, h);
  p.E = Ep;
  if (Ep <= T.eabs_g) {
    s.deposit(vox(p, R.P), Ep);
    return false;
  }
  return true;
}

// Woodcock flights until a real interaction.  With max_draws below the cap,
// a call stops after that many random draws (two flights each) and returns
// true with the photon in flight; the next call continues with the same
// random numbers, so the photon's history does not depend on the split.
template <class Real, class Ctx, class Sink>
__device__ bool photon_segment(PartT<Real> &p, const Ctx &R, Sink &s, int max_draws = kMaxPhotonFlights) {
  using N = Num<Real>;
  const auto &T = R.T;
  const auto &P = R.P;
  if (p.E <= T.eabs_g) {
    s.deposit(vox(p, P), p.E);
    return false;
  }
  const EIdxT<Real> e = eidx(T, p.E);
  const Real mumax = lerp(N::ld(P.mu_max + e.i), N::ld(P.mu_max + e.i + 1), e.f);
  const Real inv_mumax = Real(1) / mumax;
  const Real X = P.nx * P.dx, Y = P.ny * P.dy, Z = P.nz * P.dz;
  for (int it = 0; it < max_draws; ++it) {
    const uint4 r = draw(p, R);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const Real us = N::u01(j ? r.z : r.x), ua = N::u01(j ? r.w : r.y);
      s.count_flight();
      move(p, neglog(us) * inv_mumax);
      if (!(p.x >= Real(0) && p.x < X && p.y >= Real(0) && p.y < Y && p.z >= Real(0) && p.z < Z)) {
        s.escape(p.E);
        return false;
      }
      locate(p, P);
      const int v = vox(p, P);
      const int m = P.mat[v];
      const Real mu = Real(P.rho[v]) * ph_mu(T, m, e);
      if (ua * mumax < mu) {
        s.count_interaction();
        return photon_interact(p, R, s, e, m);
      }
    }
  }
  if (max_draws < kMaxPhotonFlights) return true;
  s.error(ERR_STEPCAP);
  s.deposit(vox(p, P), p.E);
  return false;
}

// ---------------------------------------------------------------------------
// Electrons and positrons (Sec. 2.1): one condensed-history step.
// Returns true while the particle is alive.
// ---------------------------------------------------------------------------
template <class Real, class Ctx, class Sink>
__device__ DPM_COLD void electron_hard(PartT<Real> &p, const Ctx &R, Sink &s, Real sig0, int m) {
  using N = Num<Real>;
  const auto &T = R.T;
  const uint4 r = draw(p, R);
  const Real Tn = p.E;
  const EIdxT<Real> e = eidx(T, Tn);
  const Real sig = el_at(T, m, e).z;
  if (N::u01(r.x) * sig0 >= sig) return;  // delta-scattering null event
  const Real pm = lerp(N::ld(T.pmol + size_t(m) * T.n_e + e.i), N::ld(T.pmol + size_t(m) * T.n_e + e.i + 1), e.f);
  const Real lnT = N::log(Tn);
  const Real ec = T.wcc / Tn;
  const Real h = Real(2) * N::u01(r.w);  // azimuth in half turns
  if (N::u01(r.y) < pm && ec < Real(0.5)) {
    // Moller: z = (1/ec - 1/eps)/(1/ec - 2)
    const Real z = samp(T.mol, lnT, N::u01(r.z));
    const Real eps = Real(1) / (Real(1) / ec - z * (Real(1) / ec - Real(2)));
    const Real W = eps * Tn, Tp = Tn - W;
    const Real cs = N::sqrt(W * (Tn + Real(2) * N::mc2) / (Tn * (W + Real(2) * N::mc2)));
    const Real cpr = N::sqrt(Tp * (Tn + Real(2) * N::mc2) / (Tn * (Tp + Real(2) * N::mc2)));
    PartT<Real> d = child(p, ELECTRON, 1);
    d.E = W;
    rotate(d.u, d.v, d.w, cs, h);
    emit_charged(d, R, s);
    rotate(p.u, p.v, p.w, cpr, h + Real(1));
    p.E = Tp;
  } else if (Tn > T.wcr) {
    // bremsstrahlung photon along the electron: y = ln(k/wcr)/ln(T/wcr)
    const Real y = samp(T.brem, lnT, N::u01(r.z));
    const Real kk = N::min(T.wcr * N::exp(y * N::log(Tn / T.wcr)), Tn);
    PartT<Real> g = child(p, PHOTON, 1);
    g.E = kk;
    emit_photon(g, R, s);
    p.E = Tn - kk;
  }
}

template <class Real, class Ctx, class Sink>
__device__ bool electron_step(PartT<Real> &p, const Ctx &R, Sink &s) {
  using N = Num<Real>;
  const auto &T = R.T;
  const auto &P = R.P;
  if (p.E <= T.eabs_e) {
    absorb_charged(p, R, s);
    return false;
  }
  s.count_step();
  const int v = vox(p, P);
  const int m = P.mat[v];
  const Real rho = P.rho[v];
  const Real T0 = p.E;
  // on the ln(E) grid the step's end energy (1 - f_e) T0, or eabs_e, lies a
  // fixed shift below T0's position: one logarithm serves both lookups
  Real x0 = egrid(T, T0);
  const Real xe = N::max(x0 + T.x_fe, T.x_eabs);
  const Real Tend = N::max((Real(1) - T.f_e) * T0, T.eabs_e);
  const typename Vec4<Real>::type r0 = el_at(T, m, eidx_x(T, x0));  // R, S, Sigma_hard, 1/lambda1
  const Real Rend = el_range(T, m, eidx_x(T, xe));
  const Real sE = N::div_hw(N::max(r0.x - Rend, Real(0)), rho);  // path lengths: hardware division (2 ulp)
  const uint4 rn = draw(p, R);
  const Real sh =
      (r0.z > Real(0) && !(T.flags & DPM_NO_HARD)) ? N::div_hw(neglog(N::u01(rn.x)), rho * r0.z) : N::inf;
  const bool hard = sh < sE;
  const Real st = hard ? sh : sE;
  const Real tau = N::u01(rn.y);
  int axis;
  bool crossed;
  Real path;
  const Real t1 = dist_to_face(p, P, axis);
  if (t1 <= tau * st) {
    move(p, t1);
    path = t1;
    crossed = true;
  } else {
    const Real th = tau * st;
    move(p, th);
    if (!(T.flags & DPM_NO_MSC)) {
      const Real A = msc_A(T, rho * st * r0.w);
      const Real omc = msc_sample(A, N::u01(rn.z));
      rotate(p.u, p.v, p.w, Real(1) - omc, Real(2) * N::u01(rn.w));
    }
    const Real rest = st - th;
    const Real t2 = dist_to_face(p, P, axis);
    if (t2 <= rest) {
      move(p, t2);
      path = th + t2;
      crossed = true;
    } else {
      move(p, rest);
      path = st;
      crossed = false;
    }
  }
  const Real Tn = (!crossed && !hard) ? Tend : csda_energy(T, m, T0, r0.x, r0.y, rho * path);
  s.deposit(v, T0 - Tn);
  p.E = Tn;
  if (crossed) {
    if (!cross_face(p, P, axis)) {
      s.escape(Tn + (p.type == POSITRON ? Real(2) * N::mc2 : Real(0)));
      return false;
    }
    return true;
  }
  if (Tn <= T.eabs_e) {
    absorb_charged(p, R, s);
    return false;
  }
  if (hard) electron_hard(p, R, s, r0.z, m);
  return true;
}

}  // namespace dpm
