// SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the output function applied to coordinates, a
// position-keyed uniform value that does not depend on the DoF numbering.
#pragma once

#include <cmath>
#include <cstdint>

namespace gcmg {

inline uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// uniform value in [-1, 1) attached to the point xyz: every coordinate is
// rounded to a multiple of 2^-20 and mixed into the state in turn
inline double point_value(const double* xyz, uint64_t seed) {
  uint64_t h = seed;
  for (int d = 0; d < 3; ++d) {
    const int64_t q = (int64_t)std::nearbyint(xyz[d] * 1048576.0);
    h ^= (uint64_t)q;
    h += 0x9E3779B97F4A7C15ull;
    h = splitmix64_mix(h);
  }
  return -1.0 + 2.0 * (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

// seed of the perturbation of the eigenvalue estimate's start vector
constexpr uint64_t LANCZOS_START_SEED = 2203;

}  // namespace gcmg
