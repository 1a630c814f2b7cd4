// k_f32.cu -- kernels whose coefficients are stored as float.
#include <algorithm>

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

// the fold kernels of the adjoint (this translation unit alone defines them);
// a level's first fold is a plain launch after its units, the folds of its
// later groups (other images) programmatic dependents of the one before
__global__ void __launch_bounds__(256) adj_fold_kernel(const InvParams p) {
    const int n = adj_fold_count(p.h, p.w);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int r, c;
        adj_fold_index(p.h, p.w, i, r, c);
        adj_fold_pixel(p, r, c);
    }
}

__global__ void __launch_bounds__(256) adj_fold_group_kernel(const __grid_constant__ InvGroupLaunch L) {
    griddep_launch_dependents();
    for (int k = blockIdx.y; k < L.n_img; k += gridDim.y) {
        const InvParams& p = L.img[k].p;
        const int n = adj_fold_count(p.h, p.w);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            int r, c;
            adj_fold_index(p.h, p.w, i, r, c);
            adj_fold_pixel(p, r, c);
        }
    }
}

namespace {
cudaLaunchConfig_t fold_config(dim3 grid, int pdl, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = dim3(256);
    lc.stream = s;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = pdl ? 1 : 0;
    return lc;
}
}  // namespace

int launch_adj_fold(const InvParams& p, cudaStream_t s) {
    const int n = adj_fold_count(p.h, p.w);
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t lc = fold_config(dim3((n + 255) / 256), 0, s, attr);
    return cudaLaunchKernelEx(&lc, adj_fold_kernel, p);
}

int launch_adj_fold_group(const InvGroupLaunch& g, int pdl, cudaStream_t s) {
    int n = 0;
    for (int k = 0; k < g.n_img; ++k) n = std::max(n, adj_fold_count(g.img[k].p.h, g.img[k].p.w));
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t lc = fold_config(dim3((n + 255) / 256, g.n_img), pdl, s, attr);
    return cudaLaunchKernelEx(&lc, adj_fold_group_kernel, g);
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
