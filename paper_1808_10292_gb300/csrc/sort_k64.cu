// Compiled kernel variants for 64-bit keys (radix 2^8 onesweep passes).
#include "onesweep.cuh"

namespace isort {

// lsd_entry<K, V, radix bits, threads, keys per thread, min CTAs per SM>;
// variant 0 is the built-in default.
static const LsdEntry kK64None8[] = {
    lsd_entry<uint64_t, NoVal, 8, 256, 20, 3>(),  // 5120-key tiles, 3 CTAs/SM
    lsd_entry<uint64_t, NoVal, 8, 512, 10, 3>(),  // 5120-key tiles, 48 warps/SM
    lsd_entry<uint64_t, NoVal, 8, 384, 16, 2>(),
    lsd_entry<uint64_t, NoVal, 8, 256, 16, 3>(),
    lsd_entry<uint64_t, NoVal, 8, 256, 24, 2>(),
};
static const LsdEntry kK64V32_8[] = {
    lsd_entry<uint64_t, uint32_t, 8, 256, 16, 2>(),
    lsd_entry<uint64_t, uint32_t, 8, 256, 16, 3>(),
    lsd_entry<uint64_t, uint32_t, 8, 256, 12, 3>(),
};
static const LsdEntry kK64V64_8[] = {
    lsd_entry<uint64_t, uint64_t, 8, 256, 12, 2>(),
    lsd_entry<uint64_t, uint64_t, 8, 256, 12, 3>(),
};

int lsd_variants_k64(int val_bits, int radix_bits, const LsdEntry** out) {
  if (radix_bits != 8) return 0;
  switch (val_bits) {
    case 0: *out = kK64None8; return (int)(sizeof(kK64None8) / sizeof(LsdEntry));
    case 32: *out = kK64V32_8; return (int)(sizeof(kK64V32_8) / sizeof(LsdEntry));
    case 64: *out = kK64V64_8; return (int)(sizeof(kK64V64_8) / sizeof(LsdEntry));
  }
  return 0;
}

}  // namespace isort
