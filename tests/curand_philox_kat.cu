// Known-answer source for the oracle's Philox4x32-10: the cuRAND header's own
// curand_Philox4x32_10(counter, key), compiled as host code (the header takes
// its host branch when QUALIFIERS names __host__) and called, never restated.
// Reads lines "c0 c1 c2 c3 k0 k1" (decimal uint32) from stdin and prints the
// four output words per line.
#define QUALIFIERS static inline __host__ __device__
#include <curand_philox4x32_x.h>
#include <cstdio>

int main() {
  unsigned c0, c1, c2, c3, k0, k1;
  while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    uint4 c = make_uint4(c0, c1, c2, c3);
    uint2 k = make_uint2(k0, k1);
    uint4 o = curand_Philox4x32_10(c, k);
    std::printf("%u %u %u %u\n", o.x, o.y, o.z, o.w);
  }
  return 0;
}
