// k_i32.cu -- kernels whose coefficients are stored as int.
#include "launch.cuh"

namespace dwt2 {

int launch_forward_i32(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p,
                   int grid, const FwdCfg& cfg, cudaStream_t s) {
    return launch_forward_t<int>(wav, scheme, box, row, p, grid, cfg, s);
}

int launch_inverse_i32(int wav, int scheme, const InvParams& p, int grid, cudaStream_t s) {
    return launch_inverse_t<int>(wav, scheme, p, grid, s);
}

int occupancy_forward_i32(int wav, int scheme, const FwdCfg& cfg) { return occupancy_forward_t<int>(wav, scheme, cfg); }
int occupancy_inverse_i32(int scheme) { return occupancy_inverse_t<int>(scheme); }

}  // namespace dwt2
