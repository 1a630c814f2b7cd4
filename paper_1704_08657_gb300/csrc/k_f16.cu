// k_f16.cu -- kernels whose coefficients are stored as __half.
#include "launch.cuh"

namespace dwt2 {

int launch_forward_f16(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p,
                   int grid, const FwdCfg& cfg, cudaStream_t s) {
    return launch_forward_t<__half>(wav, scheme, box, row, p, grid, cfg, s);
}

int launch_inverse_f16(int wav, int scheme, const InvParams& p, int grid, int pdl, int cls, cudaStream_t s) {
    return launch_inverse_t<__half>(wav, scheme, p, grid, pdl, cls, s);
}

int launch_inv_group_f16(int wav, int scheme, const InvGroupLaunch& g, int grid, int pdl, int cls, cudaStream_t s) {
    return launch_inv_group_t<__half>(wav, scheme, g, grid, pdl, cls, s);
}

int occupancy_forward_f16(int wav, int scheme, const FwdCfg& cfg) { return occupancy_forward_t<__half>(wav, scheme, cfg); }
int occupancy_inverse_f16(int wav, int scheme) { return occupancy_inverse_t<__half>(wav, scheme); }

int launch_pml_f16(int wav, int scheme, const PmlLaunch& p, int grid, cudaStream_t s) {
    return launch_pml_t<__half>(wav, scheme, &p, grid, s, false);
}
int occupancy_pml_f16(int wav, int scheme) { return launch_pml_t<__half>(wav, scheme, nullptr, 0, nullptr, true); }

int launch_fused_f16(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FusedParams& p,
                     int grid, cudaStream_t s) {
    return launch_fused_t<__half>(wav, scheme, &box, &row, &p, grid, s, false);
}
int occupancy_fused_f16(int wav, int scheme) {
    return launch_fused_t<__half>(wav, scheme, nullptr, nullptr, nullptr, 0, nullptr, true);
}

int launch_group_f16(int wav, int scheme, const GroupLaunch& g, int grid, const FwdCfg& cfg, int pdl, cudaStream_t s) {
    return launch_group_t<__half>(wav, scheme, g, grid, cfg, pdl, s);
}

}  // namespace dwt2
