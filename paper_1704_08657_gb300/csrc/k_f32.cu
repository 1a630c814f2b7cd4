// k_f32.cu -- kernels whose coefficients are stored as float.
#include "launch.cuh"

namespace dwt2 {

int launch_forward_f32(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p,
                   int grid, const FwdCfg& cfg, cudaStream_t s) {
    return launch_forward_t<float>(wav, scheme, box, row, p, grid, cfg, s);
}

int launch_inverse_f32(int wav, int scheme, const InvParams& p, int grid, int pdl, int cls, cudaStream_t s) {
    return launch_inverse_t<float>(wav, scheme, p, grid, pdl, cls, s);
}

int launch_inv_group_f32(int wav, int scheme, const InvGroupLaunch& g, int grid, int pdl, int cls, cudaStream_t s) {
    return launch_inv_group_t<float>(wav, scheme, g, grid, pdl, cls, s);
}

int occupancy_forward_f32(int wav, int scheme, const FwdCfg& cfg) { return occupancy_forward_t<float>(wav, scheme, cfg); }
int occupancy_inverse_f32(int wav, int scheme) { return occupancy_inverse_t<float>(wav, scheme); }

int launch_pml_f32(int wav, int scheme, const PmlLaunch& p, int grid, cudaStream_t s) {
    return launch_pml_t<float>(wav, scheme, &p, grid, s, false);
}
int occupancy_pml_f32(int wav, int scheme) { return launch_pml_t<float>(wav, scheme, nullptr, 0, nullptr, true); }

int launch_fused_f32(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FusedParams& p,
                     int grid, cudaStream_t s) {
    return launch_fused_t<float>(wav, scheme, &box, &row, &p, grid, s, false);
}
int occupancy_fused_f32(int wav, int scheme) {
    return launch_fused_t<float>(wav, scheme, nullptr, nullptr, nullptr, 0, nullptr, true);
}

int launch_group_f32(int wav, int scheme, const GroupLaunch& g, int grid, const FwdCfg& cfg, int pdl, cudaStream_t s) {
    return launch_group_t<float>(wav, scheme, g, grid, cfg, pdl, s);
}

}  // namespace dwt2

namespace dwt2 {

int launch_adjoint_f32(const InvParams& p, int grid, int pdl, int cls, cudaStream_t s) {
    return launch_inv_one<Adj97<INV_QL>, float, true>(p, grid, pdl, cls, s);
}

int occupancy_forward_f16(int wav, int scheme, const FwdCfg& cfg);
int occupancy_forward_bf16(int wav, int scheme, const FwdCfg& cfg);
int occupancy_forward_i32(int wav, int scheme, const FwdCfg& cfg);
int occupancy_inverse_f16(int wav, int scheme);
int occupancy_inverse_bf16(int wav, int scheme);
int occupancy_inverse_i32(int wav, int scheme);

int forward_blocks_per_sm(int wav, int scheme, int coef_dtype, const FwdCfg& cfg) {
    switch (coef_dtype) {
        case DT_F32: return occupancy_forward_f32(wav, scheme, cfg);
        case DT_F16: return occupancy_forward_f16(wav, scheme, cfg);
        case DT_BF16: return occupancy_forward_bf16(wav, scheme, cfg);
        default: return occupancy_forward_i32(wav, scheme, cfg);
    }
}

int launch_adj_group_f32(const InvGroupLaunch& g, int grid, int pdl, int cls, cudaStream_t s) {
    return launch_inv_group_one<Adj97<INV_QL>, float, true>(g, grid, pdl, cls, s);
}

int occupancy_pml_f16(int wav, int scheme);
int occupancy_pml_bf16(int wav, int scheme);
int occupancy_pml_i32(int wav, int scheme);

int pml_blocks_per_sm(int wav, int scheme, int coef_dtype) {
    switch (coef_dtype) {
        case DT_F32: return occupancy_pml_f32(wav, scheme);
        case DT_F16: return occupancy_pml_f16(wav, scheme);
        case DT_BF16: return occupancy_pml_bf16(wav, scheme);
        default: return occupancy_pml_i32(wav, scheme);
    }
}

int occupancy_fused_f16(int wav, int scheme);
int occupancy_fused_bf16(int wav, int scheme);
int occupancy_fused_i32(int wav, int scheme);

int fused_blocks_per_sm(int wav, int scheme, int coef_dtype) {
    switch (coef_dtype) {
        case DT_F32: return occupancy_fused_f32(wav, scheme);
        case DT_F16: return occupancy_fused_f16(wav, scheme);
        case DT_BF16: return occupancy_fused_bf16(wav, scheme);
        default: return occupancy_fused_i32(wav, scheme);
    }
}

int inverse_blocks_per_sm(int wav, int scheme, int coef_dtype, bool adjoint) {
    if (adjoint) return occupancy_inv_one<Adj97<INV_QL>, float, true>();
    switch (coef_dtype) {
        case DT_F32: return occupancy_inverse_f32(wav, scheme);
        case DT_F16: return occupancy_inverse_f16(wav, scheme);
        case DT_BF16: return occupancy_inverse_bf16(wav, scheme);
        default: return occupancy_inverse_i32(wav, scheme);
    }
}

const FwdCfg FWD_CFGS[N_FWD_CFGS] = {
#define DWT2_X(I_, QL_, QR_, NST_, NW_, SP_) {QL_, QR_, NST_, NW_, SP_},
    DWT2_FWD_CFG_LIST(DWT2_X)
#undef DWT2_X
};

size_t fwd_smem_bytes_of(const FwdCfg& c) {
    return size_t(c.nw) * c.nst * (2 * c.qr * 64 * c.ql * 4) + size_t(c.nw) * c.nst * 8;
}

}  // namespace dwt2
