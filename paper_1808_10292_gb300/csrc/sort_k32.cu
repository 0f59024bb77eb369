// Compiled kernel variants for 32-bit keys (radix 2^8 onesweep passes).
#include "onesweep.cuh"

namespace isort {

// Variant 0 is the built-in default; the autotuner may pick another per size.
// lsd_entry<K, V, radix bits, threads, keys per thread, min CTAs per SM>
static const LsdEntry kK32None8[] = {
    lsd_entry<uint32_t, NoVal, 8, 256, 32, 3>(),  // 8192-key tiles, 3 CTAs/SM
    lsd_entry<uint32_t, NoVal, 8, 512, 16, 3>(),  // 8192-key tiles, 48 warps/SM
    lsd_entry<uint32_t, NoVal, 8, 256, 24, 4>(),  // 4 CTAs/SM
    lsd_entry<uint32_t, NoVal, 8, 256, 20, 4>(),
    lsd_entry<uint32_t, NoVal, 8, 384, 32, 2>(),  // 12288-key tiles
    lsd_entry<uint32_t, NoVal, 8, 512, 24, 2>(),
    lsd_entry<uint32_t, NoVal, 8, 128, 32, 6>(),  // 6 CTAs/SM
    lsd_entry<uint32_t, NoVal, 8, 256, 16, 6>(),  // 4096-key tiles, 48 warps/SM
};
static const LsdEntry kK32V32_8[] = {
    lsd_entry<uint32_t, uint32_t, 8, 256, 20, 3>(),
    lsd_entry<uint32_t, uint32_t, 8, 384, 16, 2>(),
    lsd_entry<uint32_t, uint32_t, 8, 256, 16, 3>(),
    lsd_entry<uint32_t, uint32_t, 8, 256, 24, 2>(),
    lsd_entry<uint32_t, uint32_t, 8, 256, 16, 4>(),
};
static const LsdEntry kK32V64_8[] = {
    lsd_entry<uint32_t, uint64_t, 8, 256, 16, 2>(),
    lsd_entry<uint32_t, uint64_t, 8, 256, 16, 3>(),
    lsd_entry<uint32_t, uint64_t, 8, 256, 12, 3>(),
};

int lsd_variants_k32(int val_bits, int radix_bits, const LsdEntry** out) {
  if (radix_bits != 8) return 0;
  switch (val_bits) {
    case 0: *out = kK32None8; return (int)(sizeof(kK32None8) / sizeof(LsdEntry));
    case 32: *out = kK32V32_8; return (int)(sizeof(kK32V32_8) / sizeof(LsdEntry));
    case 64: *out = kK32V64_8; return (int)(sizeof(kK32V64_8) / sizeof(LsdEntry));
  }
  return 0;
}

}  // namespace isort
