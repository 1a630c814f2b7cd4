// k_f32.cu -- kernels whose coefficients are stored as float.
#include "launch.cuh"

namespace dwt2 {

int launch_forward_f32(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p,
                   int grid, const FwdCfg& cfg, cudaStream_t s) {
    return launch_forward_t<float>(wav, scheme, box, row, p, grid, cfg, s);
}

int launch_inverse_f32(int wav, int scheme, const InvParams& p, int grid, cudaStream_t s) {
    return launch_inverse_t<float>(wav, scheme, p, grid, s);
}

}  // namespace dwt2

namespace dwt2 {

int launch_adjoint_f32(const InvParams& p, int grid, cudaStream_t s) {
    return launch_inv_one<Adj97, float, true>(p, grid, s);
}

const FwdCfg FWD_CFGS[N_FWD_CFGS] = {
#define DWT2_X(I_, QR_, NST_, NW_) {QR_, NST_, NW_},
    DWT2_FWD_CFG_LIST(DWT2_X)
#undef DWT2_X
};

size_t fwd_smem_bytes_of(const FwdCfg& c) {
    return size_t(c.nw) * c.nst * (2 * c.qr * STRIP_PX * 4) + size_t(c.nw) * c.nst * 8;
}

}  // namespace dwt2
