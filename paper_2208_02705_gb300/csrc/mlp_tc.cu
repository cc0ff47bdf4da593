// placeholder until the tcgen05 kernel lands
#include "internal.cuh"
namespace roam {
bool tc_supported(int, int) { return false; }
int64_t tc_image_bytes(int, int) { return 0; }
int tc_bias_count(int, int) { return 0; }
int tc_tile_samples() { return 128; }
void launch_pack_tc(const float *, int, int, int, int64_t, void *, int64_t, float *, int, cudaStream_t) {}
void launch_mlp_tc(const MlpWeights &, const SampleSrc &, const BucketBufs &, Counters *, float4 *, int, cudaStream_t) {}
}  // namespace roam
