// dpm_device.cuh -- device-side transport physics (FP32), shared by the
// transport kernels.  Every function follows the DPM scheme of Sec. 2.1 with
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
#pragma once

#include <cuda_runtime.h>

#include "dpm_internal.h"

namespace dpm {

constexpr float kMc2f = 0.51099895f;
constexpr float kTwoPi = 6.283185307179586f;
constexpr float kPif = 3.141592653589793f;
constexpr float kInf = 3.0e38f;
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

// uniform on (0, 1] from the top 24 bits: (k + 1/2) 2^-24 for k = x >> 8, in
// one rounding (the top values round to 1)
__device__ __forceinline__ float u01(uint32_t x) {
  return fmaf(float(x >> 8), 1.0f / 16777216.0f, 1.0f / 33554432.0f);
}

// -ln(u) for an exponential free path, with the hardware logarithm (absolute
// error about 2^-21 near u = 1, far below the paths' statistical spread); the
// clamp keeps a rounding just above zero from reversing a flight.
__device__ __forceinline__ float neglog(float u) { return fmaxf(-__logf(u), 0.f); }

// ---------------------------------------------------------------------------
// Particle state.  (ix, iy, iz) are tracked exactly across voxel faces.
// ---------------------------------------------------------------------------
enum : int { PHOTON = 0, ELECTRON = 1, POSITRON = 2 };

struct Part {
  float x, y, z, u, v, w, E;
  int ix, iy, iz;
  uint32_t id_lo, id_hi;  // particle id within its history
  uint32_t ctr;           // next Philox block of this particle
  uint32_t hist;          // history index relative to the run (or job)
  int type;
  int job;                // index in the batch's job table (0 for a single run)
};

// Philox key of a history: seed hash xor the global history id; the third
// counter word carries more seed bits so that different seeds never share
// streams.
template <class Ctx>
__device__ __forceinline__ uint4 draw(Part &p, const Ctx &R) {
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
__device__ __forceinline__ Part child(const Part &p, int type, uint32_t ordinal) {
  Part c = p;
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
__device__ __forceinline__ int vox(const Part &p, const DevPhantom &P) { return p.ix + P.nx * (p.iy + P.ny * p.iz); }

// Path length to the next face along one axis.  The hardware division (2 ulp)
// suffices: a step that reaches a face puts the coordinate on the face
// exactly (cross_face), so its error only moves the step length by 2 ulp.
__device__ __forceinline__ float face_dist(float x, float u, int i, float d) {
  if (u > 0.f) return fmaxf(__fdividef(fmaf(float(i + 1), d, -x), u), 0.f);
  if (u < 0.f) return fmaxf(__fdividef(fmaf(float(i), d, -x), u), 0.f);
  return kInf;
}

__device__ __forceinline__ float dist_to_face(const Part &p, const DevPhantom &P, int &axis) {
  float t = face_dist(p.x, p.u, p.ix, P.dx);
  axis = 0;
  const float ty = face_dist(p.y, p.v, p.iy, P.dy);
  if (ty < t) { t = ty; axis = 1; }
  const float tz = face_dist(p.z, p.w, p.iz, P.dz);
  if (tz < t) { t = tz; axis = 2; }
  return t;
}

__device__ __forceinline__ void move(Part &p, float s) {
  p.x = fmaf(s, p.u, p.x);
  p.y = fmaf(s, p.v, p.y);
  p.z = fmaf(s, p.w, p.z);
}

// Step into the neighbour across `axis`; false if that leaves the phantom.
__device__ __forceinline__ bool cross_face(Part &p, const DevPhantom &P, int axis) {
  if (axis == 0) {
    if (p.u > 0.f) { p.ix += 1; p.x = float(p.ix) * P.dx; } else { p.x = float(p.ix) * P.dx; p.ix -= 1; }
    return p.ix >= 0 && p.ix < P.nx;
  }
  if (axis == 1) {
    if (p.v > 0.f) { p.iy += 1; p.y = float(p.iy) * P.dy; } else { p.y = float(p.iy) * P.dy; p.iy -= 1; }
    return p.iy >= 0 && p.iy < P.ny;
  }
  if (p.w > 0.f) { p.iz += 1; p.z = float(p.iz) * P.dz; } else { p.z = float(p.iz) * P.dz; p.iz -= 1; }
  return p.iz >= 0 && p.iz < P.nz;
}

// Voxel containing a point known to be inside the phantom.
__device__ __forceinline__ void locate(Part &p, const DevPhantom &P) {
  p.ix = min(max(int(floorf(p.x / P.dx)), 0), P.nx - 1);
  p.iy = min(max(int(floorf(p.y / P.dy)), 0), P.ny - 1);
  p.iz = min(max(int(floorf(p.z / P.dz)), 0), P.nz - 1);
}

// Rotate the direction by polar cosine c and azimuth pi*h (h in half turns).
// h is reduced modulo 2 to [-1, 1), where the hardware sine and cosine are
// accurate to about 2^-21 absolute; the direction is renormalised below.
__device__ __forceinline__ void rotate(float &u, float &v, float &w, float c, float h) {
  c = fminf(fmaxf(c, -1.f), 1.f);
  const float c2 = fmaxf(0.f, fmaf(-c, c, 1.f));
  const float s = c2 * rsqrtf(fmaxf(c2, 1e-30f));  // sin(theta) by the hardware 1/sqrt
  float sp, cp;
  const float t = h - 2.f * floorf(0.5f * h + 0.5f);  // h modulo 2, in [-1, 1)
  __sincosf(3.14159265f * t, &sp, &cp);
  const float r2 = fmaf(u, u, v * v);
  float nu, nv, nw;
  if (r2 < 1e-10f) {
    nu = s * cp;
    nv = s * sp;
    nw = (w >= 0.f) ? c : -c;
  } else {
    const float ir = rsqrtf(r2), r = r2 * ir, a = s * ir;  // hardware 1/sqrt; renormalised below
    nu = fmaf(u, c, a * fmaf(u * w, cp, -(v * sp)));
    nv = fmaf(v, c, a * fmaf(v * w, cp, u * sp));
    nw = fmaf(w, c, -(s * r) * cp);
  }
  const float n = rsqrtf(fmaf(nu, nu, fmaf(nv, nv, nw * nw)));
  u = nu * n;
  v = nv * n;
  w = nw * n;
}

// ---------------------------------------------------------------------------
// Table access: linear interpolation on a uniform ln(E) grid
// ---------------------------------------------------------------------------
struct EIdx {
  int i;
  float f;
};

// Grid position x (fractional node index) clamped to the table.
__device__ __forceinline__ EIdx eidx_x(const DevTables &T, float x) {
  x = fminf(fmaxf(x, 0.f), float(T.n_e - 1) - 1e-3f);
  EIdx e;
  e.i = int(x);
  e.f = x - float(e.i);
  return e;
}

// Fractional node index of energy E on the uniform ln E grid, from the
// hardware base-2 logarithm in one FMA (x_lg2 = ln 2 / spacing, x_lo = -ln E_lo
// / spacing).  The intrinsic's documented error (2 ulp of log2 E, within
// 7e-7 of ln E on the tables' range) moves the position by at most 2.5e-4 of
// a node spacing at 2048 nodes: an interpolation error well below the
// tables' own.
__device__ __forceinline__ float egrid(const DevTables &T, float E) { return fmaf(__log2f(E), T.x_lg2, T.x_lo); }

__device__ __forceinline__ EIdx eidx(const DevTables &T, float E) {
  float x = egrid(T, E);
  x = fminf(fmaxf(x, 0.f), float(T.n_e - 1) - 1e-3f);
  EIdx e;
  e.i = int(x);
  e.f = x - float(e.i);
  return e;
}

__device__ __forceinline__ float lerp(float a, float b, float f) { return fmaf(f, b - a, a); }

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float f) {
  return make_float4(lerp(a.x, b.x, f), lerp(a.y, b.y, f), lerp(a.z, b.z, f), lerp(a.w, b.w, f));
}

// The per-material float4 tables hold, for every node, its value and the
// difference to the next node (a 32-byte record): one interpolation reads one
// aligned sector and takes one FMA per component, with the same result as
// interpolating between the two nodes (the difference is the same float
// subtraction, done when the table is uploaded).
__device__ __forceinline__ float4 lerp_node(const float4 *b, float f) {
  const float4 v = __ldg(b), d = __ldg(b + 1);
  return make_float4(fmaf(f, d.x, v.x), fmaf(f, d.y, v.y), fmaf(f, d.z, v.z), fmaf(f, d.w, v.w));
}

__device__ __forceinline__ float lerp_node_x(const float4 *b, float f) {
  return fmaf(f, __ldg(&b[1].x), __ldg(&b[0].x));
}

__device__ __forceinline__ float4 el_at(const DevTables &T, int m, EIdx e) {
  return lerp_node(T.el + 2 * (size_t(m) * T.n_e + e.i), e.f);
}

__device__ __forceinline__ float el_range(const DevTables &T, int m, EIdx e) {
  return lerp_node_x(T.el + 2 * (size_t(m) * T.n_e + e.i), e.f);
}

__device__ __forceinline__ float4 ph_at(const DevTables &T, int m, EIdx e) {
  return lerp_node(T.ph + 2 * (size_t(m) * T.n_e + e.i), e.f);
}

__device__ __forceinline__ float ph_mu(const DevTables &T, int m, EIdx e) {
  return lerp_node_x(T.ph + 2 * (size_t(m) * T.n_e + e.i), e.f);
}

__device__ __forceinline__ float samp(const SampTab &t, float lnE, float u) {
  float x = (lnE - t.lnE0) * t.inv_dlnE;
  x = fminf(fmaxf(x, 0.f), float(t.ne - 1) - 1e-3f);
  const int i = int(x);
  const float fx = x - float(i);
  const float yk = u * float(t.nu - 1);
  const int k = min(int(yk), t.nu - 2);
  const float fy = yk - float(k);
  const float *r0 = t.y + size_t(i) * t.nu + k;
  const float a = lerp(__ldg(r0), __ldg(r0 + 1), fy);
  const float b = lerp(__ldg(r0 + t.nu), __ldg(r0 + t.nu + 1), fy);
  return lerp(a, b, fx);
}

// A of the random-hinge distribution for a step of x = s/lambda1: the table is
// ln A against logit(q), q = 1 - exp(-x); beyond its ends ln A grows like logit(q).
__device__ __forceinline__ float msc_A(const DevTables &T, float x) {
  // q = 1 - exp(-x): a Taylor polynomial below x = 0.1 (truncation under
  // 1e-7 relative), the hardware exponential above (2 ulp of exp(-x), at
  // most 3e-6 of q); the hardware logarithm then moves the table position
  // by a few 1e-6
  const float q = x < 0.1f ? x * fmaf(-x, fmaf(-x, fmaf(-x, 1.f / 24.f, 1.f / 6.f), 0.5f), 1.f) : 1.f - __expf(-x);
  const float lg = __logf(q) + x;
  const float t = (lg - T.msc_x0) * T.msc_inv_dx;
  float lA;
  if (!(t > 0.f)) {  // also catches NaN
    lA = __ldg(T.msc_lnA) + (lg - T.msc_x0);
  } else if (t >= float(T.msc_n - 1)) {
    lA = __ldg(T.msc_lnA + T.msc_n - 1) + (lg - (T.msc_x0 + float(T.msc_n - 1) / T.msc_inv_dx));
  } else {
    const int i = int(t);
    lA = lerp(__ldg(T.msc_lnA + i), __ldg(T.msc_lnA + i + 1), t - float(i));
  }
  return __expf(fminf(lA, 60.f));  // hardware exponential: a few ulp at the ln A of real steps
}

// 1 - mu of the hinge distribution by its inverse CDF (hardware division,
// 2 ulp: far below the table's interpolation error).
__device__ __forceinline__ float msc_sample(float A, float xi) { return __fdividef(2.f * A * xi, 1.f + A - xi); }

// Kinetic energy after a CSDA mass path mp from T0 (range R0, stopping power S0
// at T0): Euler estimate refined by one Newton step on the range table.  For
// a step losing at most 5 % of T the Euler error is about (dT)^2 |S'|/(2S);
// the Newton step squares it, to about 1e-4 of the step's loss at 0.2 MeV
// and far less above.  A second step (one more dependent table load on the
// electron's critical path) measured 2-4 % slower.
__device__ __forceinline__ float csda_energy(const DevTables &T, int m, float T0, float R0, float S0, float mp) {
  const float Rt = R0 - mp;
  const float T1 = fmaxf(fmaf(-mp, S0, T0), 0.5f * T0);
  const float4 r = el_at(T, m, eidx(T, T1));
  return fminf(fmaf(-(r.x - Rt), r.y, T1), T0);
}

// Synthetic 6 MV spectrum f(E) ~ (1 - E/6) E^-1/2 on [0.25, 6] MeV: the CDF in
// t = sqrt(E) is the cubic 2t - t^3/9; its middle root by the trigonometric
// formula.
__device__ __forceinline__ float spectrum_6mv(float u) {
  const float F0 = 0.98611111f;  // 2(0.5) - 0.5^3/9
  const float F1 = 3.26598632f;  // 2 sqrt6 - 6 sqrt6/9
  const float c = F0 + u * (F1 - F0);
  const float arg = fminf(fmaxf(-0.30618622f * c, -1.f), 1.f);  // -(3/4) c / sqrt(6)
  const float t = 4.89897949f * cosf(acosf(arg) * (1.f / 3.f) - 2.09439510f);
  return fminf(fmaxf(t * t, 0.25f), 6.0f);
}

// ---------------------------------------------------------------------------
// Emission helpers: below the absorption energy a new particle deposits on the
// spot (Sec. 3); a positron then also annihilates.
// ---------------------------------------------------------------------------
template <class Ctx, class Sink>
__device__ DPM_COLD void annihilate(Part &p, const Ctx &R, Sink &s) {
  const uint4 r = draw(p, R);
  const float cz = 2.f * u01(r.x) - 1.f;
  const float sz = sqrtf(fmaxf(0.f, 1.f - cz * cz));
  float sp, cp;
  sincospif(2.f * u01(r.y), &sp, &cp);
  Part g = child(p, PHOTON, 1);
  g.E = kMc2f;
  g.u = sz * cp;
  g.v = sz * sp;
  g.w = cz;
  s.push(g);
  Part h = child(p, PHOTON, 2);
  h.E = kMc2f;
  h.u = -g.u;
  h.v = -g.v;
  h.w = -g.w;
  s.push(h);
}

template <class Ctx, class Sink>
__device__ void emit_charged(Part &q, const Ctx &R, Sink &s) {
  if (q.E > R.T.eabs_e) {
    s.push(q);
    return;
  }
  s.deposit(vox(q, R.P), q.E);
  if (q.type == POSITRON) annihilate(q, R, s);
}

template <class Ctx, class Sink>
__device__ void emit_photon(Part &q, const Ctx &R, Sink &s) {
  if (q.E > R.T.eabs_g) s.push(q);
  else s.deposit(vox(q, R.P), q.E);
}

template <class Ctx, class Sink>
__device__ void absorb_charged(Part &p, const Ctx &R, Sink &s) {
  s.deposit(vox(p, R.P), p.E);
  if (p.type == POSITRON) annihilate(p, R, s);
}

// ---------------------------------------------------------------------------
// Source (Sec. 3): point source at SAD from the isocentre, uniform over the
// field rectangle in the isocentre plane, flown to the phantom surface.
// Returns false if the ray misses the phantom.
// ---------------------------------------------------------------------------
template <class Ctx>
__device__ DPM_COLD bool make_primary(Part &p, const Ctx &R, uint32_t hl) {
  const DevSource &S = R.S;
  const DevPhantom &P = R.P;
  p.hist = hl;
  p.job = 0;
  p.id_lo = 1u;
  p.id_hi = 0u;
  p.ctr = 0;
  p.type = (S.particle == 0) ? PHOTON : ELECTRON;
  const uint4 r = draw(p, R);
  const float a = (u01(r.x) - 0.5f) * S.fx, b = (u01(r.y) - 0.5f) * S.fy;
  float dx = S.cx + a * S.e1x - S.sx, dy = S.cy + b - S.sy, dz = S.cz + a * S.e1z - S.sz;
  const float n = rsqrtf(dx * dx + dy * dy + dz * dz);
  dx *= n;
  dy *= n;
  dz *= n;
  p.E = (S.spectrum == 1) ? spectrum_6mv(u01(r.z)) : S.energy;
  const float L[3] = {P.nx * P.dx, P.ny * P.dy, P.nz * P.dz};
  const float o[3] = {S.sx, S.sy, S.sz}, d[3] = {dx, dy, dz};
  float t0 = 0.f, t1 = kInf;
  int face = -1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (d[k] == 0.f) {
      if (o[k] < 0.f || o[k] > L[k]) return false;
      continue;
    }
    float ta = (0.f - o[k]) / d[k], tb = (L[k] - o[k]) / d[k];
    if (ta > tb) { const float t = ta; ta = tb; tb = t; }
    if (ta > t0) { t0 = ta; face = k; }
    t1 = fminf(t1, tb);
  }
  if (!(t1 > t0)) return false;
  p.x = fmaf(t0, dx, S.sx);
  p.y = fmaf(t0, dy, S.sy);
  p.z = fmaf(t0, dz, S.sz);
  p.u = dx;
  p.v = dy;
  p.w = dz;
  if (face == 0) p.x = dx > 0.f ? 0.f : L[0];
  if (face == 1) p.y = dy > 0.f ? 0.f : L[1];
  if (face == 2) p.z = dz > 0.f ? 0.f : L[2];
  locate(p, P);
  return true;
}

// ---------------------------------------------------------------------------
// Photons (Sec. 2.1): Woodcock flights over the majorant, then an interaction.
// Returns true while the photon is alive (after a Compton scatter).
// ---------------------------------------------------------------------------
template <class Ctx, class Sink>
__device__ DPM_COLD bool photon_interact(Part &p, const Ctx &R, Sink &s, EIdx e, int m) {
  const DevTables &T = R.T;
  const uint4 r = draw(p, R);
  const float4 c = ph_at(T, m, e);
  const float u0 = u01(r.x);
  const float E = p.E, k = E / kMc2f, lnE = logf(E);
  bool pair = u0 >= c.y + c.z;
  float lo = 0.f, hi = 0.f;
  if (pair) {
    const float disc = 1.f - 3.29744254f / k;  // 2 e^{1/2} / k
    if (k <= 2.f || disc <= 0.f) {
      pair = false;  // below the model's threshold (interpolation edge): scatter instead
    } else {
      const float sq = sqrtf(disc);
      lo = fmaxf(1.f / k, 0.5f * (1.f - sq));
      hi = fminf(1.f - 1.f / k, 0.5f * (1.f + sq));
      if (!(hi > lo)) pair = false;
    }
  }
  if (!pair && u0 >= c.y && u0 < c.y + c.z) {
    // photoelectric absorption: the electron takes the photon energy and direction
    Part el = child(p, ELECTRON, 1);
    emit_charged(el, R, s);
    return false;
  }
  if (pair) {
    const float eps = lo + samp(T.pair, lnE, u01(r.y)) * (hi - lo);
    Part a = child(p, ELECTRON, 1), b = child(p, POSITRON, 2);
    a.E = fmaxf(eps * E - kMc2f, 0.f);
    b.E = fmaxf((1.f - eps) * E - kMc2f, 0.f);
    emit_charged(a, R, s);
    emit_charged(b, R, s);
    return false;
  }
  // Compton (Klein-Nishina): y = ln(eps)/ln(eps0)
  const float l0 = -log1pf(2.f * k);
  const float eps = expf(samp(T.kn, lnE, u01(r.y)) * l0);
  const float Ep = eps * E, Te = E - Ep;
  const float cth = 1.f - (1.f / eps - 1.f) / k;
  const float h = 2.f * u01(r.z);  // azimuth in half turns
  Part el = child(p, ELECTRON, 1);
  el.E = Te;
  const float pe = sqrtf(Te * (Te + 2.f * kMc2f));
  const float ce = pe > 0.f ? (E - Ep * cth) / pe : 1.f;
  rotate(el.u, el.v, el.w, ce, h + 1.f);
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
template <class Ctx, class Sink>
__device__ bool photon_segment(Part &p, const Ctx &R, Sink &s, int max_draws = kMaxPhotonFlights) {
  const DevTables &T = R.T;
  const DevPhantom &P = R.P;
  if (p.E <= T.eabs_g) {
    s.deposit(vox(p, P), p.E);
    return false;
  }
  const EIdx e = eidx(T, p.E);
  const float mumax = lerp(__ldg(P.mu_max + e.i), __ldg(P.mu_max + e.i + 1), e.f);
  const float inv_mumax = 1.f / mumax;
  const float X = P.nx * P.dx, Y = P.ny * P.dy, Z = P.nz * P.dz;
  for (int it = 0; it < max_draws; ++it) {
    const uint4 r = draw(p, R);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float us = u01(j ? r.z : r.x), ua = u01(j ? r.w : r.y);
      s.count_flight();
      move(p, neglog(us) * inv_mumax);
      if (!(p.x >= 0.f && p.x < X && p.y >= 0.f && p.y < Y && p.z >= 0.f && p.z < Z)) {
        s.escape(p.E);
        return false;
      }
      locate(p, P);
      const int v = vox(p, P);
      const int m = P.mat[v];
      const float mu = P.rho[v] * ph_mu(T, m, e);
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
template <class Ctx, class Sink>
__device__ DPM_COLD void electron_hard(Part &p, const Ctx &R, Sink &s, float sig0, int m) {
  const DevTables &T = R.T;
  const uint4 r = draw(p, R);
  const float Tn = p.E;
  const EIdx e = eidx(T, Tn);
  const float sig = el_at(T, m, e).z;
  if (u01(r.x) * sig0 >= sig) return;  // delta-scattering null event
  const float pm = lerp(__ldg(T.pmol + size_t(m) * T.n_e + e.i), __ldg(T.pmol + size_t(m) * T.n_e + e.i + 1), e.f);
  const float lnT = logf(Tn);
  const float ec = T.wcc / Tn;
  const float h = 2.f * u01(r.w);  // azimuth in half turns
  if (u01(r.y) < pm && ec < 0.5f) {
    // Moller: z = (1/ec - 1/eps)/(1/ec - 2)
    const float z = samp(T.mol, lnT, u01(r.z));
    const float eps = 1.f / (1.f / ec - z * (1.f / ec - 2.f));
    const float W = eps * Tn, Tp = Tn - W;
    const float cs = sqrtf(W * (Tn + 2.f * kMc2f) / (Tn * (W + 2.f * kMc2f)));
    const float cpr = sqrtf(Tp * (Tn + 2.f * kMc2f) / (Tn * (Tp + 2.f * kMc2f)));
    Part d = child(p, ELECTRON, 1);
    d.E = W;
    rotate(d.u, d.v, d.w, cs, h);
    emit_charged(d, R, s);
    rotate(p.u, p.v, p.w, cpr, h + 1.f);
    p.E = Tp;
  } else if (Tn > T.wcr) {
    // bremsstrahlung photon along the electron: y = ln(k/wcr)/ln(T/wcr)
    const float y = samp(T.brem, lnT, u01(r.z));
    const float kk = fminf(T.wcr * expf(y * logf(Tn / T.wcr)), Tn);
    Part g = child(p, PHOTON, 1);
    g.E = kk;
    emit_photon(g, R, s);
    p.E = Tn - kk;
  }
}

template <class Ctx, class Sink>
__device__ bool electron_step(Part &p, const Ctx &R, Sink &s) {
  const DevTables &T = R.T;
  const DevPhantom &P = R.P;
  if (p.E <= T.eabs_e) {
    absorb_charged(p, R, s);
    return false;
  }
  s.count_step();
  const int v = vox(p, P);
  const int m = P.mat[v];
  const float rho = P.rho[v];
  const float T0 = p.E;
  // on the ln(E) grid the step's end energy (1 - f_e) T0, or eabs_e, lies a
  // fixed shift below T0's position: one logarithm serves both lookups
  float x0 = egrid(T, T0);
  const float xe = fmaxf(x0 + T.x_fe, T.x_eabs);
  const float Tend = fmaxf((1.f - T.f_e) * T0, T.eabs_e);
  const float4 r0 = el_at(T, m, eidx_x(T, x0));  // R, S, Sigma_hard, 1/lambda1
  const float Rend = el_range(T, m, eidx_x(T, xe));
  const float sE = __fdividef(fmaxf(r0.x - Rend, 0.f), rho);  // path lengths: hardware division (2 ulp)
  const uint4 rn = draw(p, R);
  const float sh = (r0.z > 0.f && !(T.flags & DPM_NO_HARD)) ? __fdividef(neglog(u01(rn.x)), rho * r0.z) : kInf;
  const bool hard = sh < sE;
  const float st = hard ? sh : sE;
  const float tau = u01(rn.y);
  int axis;
  bool crossed;
  float path;
  const float t1 = dist_to_face(p, P, axis);
  if (t1 <= tau * st) {
    move(p, t1);
    path = t1;
    crossed = true;
  } else {
    const float th = tau * st;
    move(p, th);
    if (!(T.flags & DPM_NO_MSC)) {
      const float A = msc_A(T, rho * st * r0.w);
      const float omc = msc_sample(A, u01(rn.z));
      rotate(p.u, p.v, p.w, 1.f - omc, 2.f * u01(rn.w));
    }
    const float rest = st - th;
    const float t2 = dist_to_face(p, P, axis);
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
  const float Tn = (!crossed && !hard) ? Tend : csda_energy(T, m, T0, r0.x, r0.y, rho * path);
  s.deposit(v, T0 - Tn);
  p.E = Tn;
  if (crossed) {
    if (!cross_face(p, P, axis)) {
      s.escape(Tn + (p.type == POSITRON ? 2.f * kMc2f : 0.f));
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
