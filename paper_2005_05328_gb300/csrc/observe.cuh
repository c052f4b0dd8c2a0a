// observe.cuh -- binning of lightcone records into the observables (paper
// Sec. 3.1.2 sky-projected lightcone, Sec. 3.1.3 3D lightcone), shared by the
// record kernel of the step (fused: each record is binned where it is made)
// and by the entry point that bins caller-supplied records.
//
// Sky map: equal-area RING pixelisation of Górski et al. (2005), 12 Nside^2
// pixels.  In the belt |z| <= 2/3 a direction lies between the pixel edge
// lines Nside (1/2 + t) -+ (3/4) Nside z = integer (t = phi / (pi/2)); the
// two line indices give the ring and the position in the ring.  In the polar
// caps the edges are t' w = integer and (1 - t') w = integer with
// w = Nside sqrt(3 (1 - |z|)), t' = t - floor(t).  Every floating-point
// operation that decides a pixel is a correctly rounded FP64 intrinsic
// (no contraction); atan2 is CUDA's.
#pragma once

#include "common.cuh"

namespace dzs {

__device__ __forceinline__ int64_t ring_pixel(int64_t nside, double x, double y, double z) {
  const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
  const double cz = r > 0.0 ? __ddiv_rn(z, r) : 1.0;
  const double za = fabs(cz);
  double phi = (x == 0.0 && y == 0.0) ? 0.0 : atan2(y, x);
  if (phi < 0.0) phi = __dadd_rn(phi, 6.283185307179586);
  double t = __ddiv_rn(phi, 1.5707963267948966);
  if (t >= 4.0) t = __dsub_rn(t, 4.0);
  const double ns = (double)nside;
  if (za <= 2.0 / 3.0) {
    const double a = __dmul_rn(ns, __dadd_rn(0.5, t));
    const double b = __dmul_rn(__dmul_rn(ns, 0.75), cz);
    const int64_t lo = (int64_t)floor(__dsub_rn(a, b));   // edge line index, ascending
    const int64_t hi = (int64_t)floor(__dadd_rn(a, b));   // edge line index, descending
    const int64_t ring = nside + 1 + lo - hi;               // 1 .. 2 nside + 1 inside the belt
    const int64_t centred0 = 1 - (ring & 1);                // a pixel centred on phi = 0
    int64_t q = lo + hi - nside + centred0;                 // even
    q = (q >= 0 ? q : q - 1) / 2;                           // floor division by 2
    int64_t pos = q % (4 * nside);
    if (pos < 0) pos += 4 * nside;
    return 2 * nside * (nside - 1) + (ring - 1) * 4 * nside + pos;
  }
  const double tf = __dsub_rn(t, floor(t));
  const double w = __dmul_rn(ns, __dsqrt_rn(__dmul_rn(3.0, __dsub_rn(1.0, za))));
  const int64_t e1 = (int64_t)floor(__dmul_rn(tf, w));
  const int64_t e2 = (int64_t)floor(__dmul_rn(__dsub_rn(1.0, tf), w));
  const int64_t ring = e1 + e2 + 1;  // from the nearer pole, 1 .. nside
  int64_t pos = (int64_t)floor(__dmul_rn(t, (double)ring)) % (4 * ring);
  if (pos < 0) pos += 4 * ring;
  if (cz > 0.0) return 2 * ring * (ring - 1) + pos;
  return 12 * nside * nside - 2 * ring * (ring + 1) + pos;
}

__device__ __forceinline__ void observe_record(const ObserveTarget& o, uint32_t k, double a, const double x[3]) {
  if (!(a >= o.a_lo && a < o.a_hi)) return;
  if (o.sky) {
    int64_t pix = ring_pixel(o.nside, __dsub_rn(x[0], o.half), __dsub_rn(x[1], o.half), __dsub_rn(x[2], o.half));
    atomicAdd(&o.sky[pix], (unsigned long long)k);
  }
  if (o.grid) {
    int64_t c[3];
    for (int ax = 0; ax < 3; ++ax) {
      c[ax] = (int64_t)floor(__dmul_rn(__ddiv_rn(x[ax], o.box), (double)o.mesh));
      c[ax] = c[ax] < 0 ? 0 : (c[ax] >= o.mesh ? o.mesh - 1 : c[ax]);
    }
    atomicAdd(&o.grid[(c[0] * o.mesh + c[1]) * o.mesh + c[2]], (unsigned long long)k);
  }
}

}  // namespace dzs
