// Compiled segmented-sort families for 32-bit keys.
#include "segmented.cuh"

namespace isort {

// <K, V, warp M, mid M, CTA M, radix threads, keys per thread, min CTAs per SM>
static const SegConfig kSeg32[] = {
    seg_config<uint32_t, NoVal, 4, 8, 16, 256, 32, 3>(),
    seg_config<uint32_t, uint32_t, 4, 8, 16, 256, 20, 3>(),
    seg_config<uint32_t, uint64_t, 4, 8, 16, 256, 16, 2>(),
};

const SegConfig* seg_config_k32(int val_bits) {
  switch (val_bits) {
    case 0: return &kSeg32[0];
    case 32: return &kSeg32[1];
    case 64: return &kSeg32[2];
  }
  return nullptr;
}

}  // namespace isort
