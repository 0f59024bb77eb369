// Compiled segmented-sort families for 64-bit keys.
#include "segmented.cuh"

namespace isort {

// <K, V, warp M, mid M, CTA M, radix threads, keys per thread, min CTAs per SM>
static const SegConfig kSeg64[] = {
    seg_config<uint64_t, NoVal, 4, 8, 8, 256, 20, 3>(),
    seg_config<uint64_t, uint32_t, 4, 8, 8, 256, 16, 2>(),
    seg_config<uint64_t, uint64_t, 4, 8, 8, 256, 12, 2>(),
};

const SegConfig* seg_config_k64(int val_bits) {
  switch (val_bits) {
    case 0: return &kSeg64[0];
    case 32: return &kSeg64[1];
    case 64: return &kSeg64[2];
  }
  return nullptr;
}

}  // namespace isort
