// dg_k3d.cu -- placeholder until the 3D stage kernel lands.
#include "dg_internal.h"
namespace dgk {
int stage3d_variants(int) { return 1; }
const char* stage3d_variant_name(int, int) { return "none"; }
cudaError_t launch_stage3d(int, int, const Stage3DArgs<double>&, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_stage3d(int, int, const Stage3DArgs<float>&, cudaStream_t) { return cudaErrorNotSupported; }
}
