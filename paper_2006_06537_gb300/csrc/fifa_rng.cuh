// Device-side Philox4x32-10, uniforms, Box-Muller normals and the
// Marsaglia-Tsang (2000) gamma sampler (see k_vec.cu for the definitions).
#pragma once
#include <stdint.h>

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ double u52(uint32_t a, uint32_t b) {
  const uint64_t k = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
  return ((double)k + 0.5) * 0x1p-52;
}

__device__ __forceinline__ uint4 philox_call(uint64_t seed, uint32_t idx, uint32_t tag, uint64_t it, uint64_t sid) {
  return philox4x32_10(make_uint4(idx, tag, (uint32_t)it, (uint32_t)sid), (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ void philox_normal_pair(uint64_t seed, uint32_t idx, uint32_t tag, uint64_t it, uint64_t sid,
                                                   double& z0, double& z1) {
  const uint4 w = philox_call(seed, idx, tag, it, sid);
  const double u0 = u52(w.x, w.y), u1 = u52(w.z, w.w);
  const double rad = sqrt(-2.0 * log(u0));
  double sn, cs;
  sincos((2.0 * 3.141592653589793) * u1, &sn, &cs);
  z0 = rad * cs;
  z1 = rad * sn;
}

__device__ __forceinline__ double philox_normal(uint64_t seed, uint32_t idx, uint32_t tag, uint64_t it, uint64_t sid) {
  double z0, z1;
  philox_normal_pair(seed, idx, tag, it, sid, z0, z1);
  return z0;
}

__device__ __forceinline__ double philox_uniform(uint64_t seed, uint32_t idx, uint32_t tag, uint64_t it, uint64_t sid) {
  const uint4 w = philox_call(seed, idx, tag, it, sid);
  return u52(w.x, w.y);
}

// Gamma(alpha, 1), alpha >= 1: attempt t uses counters 2t (normal), 2t+1 (uniform).
__device__ inline double gamma_mt(double alpha, uint64_t seed, uint32_t tag, uint64_t it, uint64_t sid) {
  const double d = alpha - 1.0 / 3.0;
  const double c = 1.0 / sqrt(9.0 * d);
  for (int t = 0; t < 64; ++t) {
    const double z = philox_normal(seed, 2u * t, tag, it, sid);
    const double u = philox_uniform(seed, 2u * t + 1u, tag, it, sid);
    double v = 1.0 + c * z;
    if (v <= 0.0) continue;
    v = v * v * v;
    if (log(u) < 0.5 * z * z + d - d * v + d * log(v)) return d * v;
  }
  return d;
}
