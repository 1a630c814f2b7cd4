// launch.cuh -- kernel instantiation and launch helpers; included by one
// translation unit per coefficient type.
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace dwt2 {

template <class Pipe, class OutT, int QR, int NST, int NW>
int launch_fwd_one(const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p, int grid, cudaStream_t s) {
    auto k = fwd_tma_kernel<Pipe, OutT, QR, NST, NW>;
    constexpr size_t smem = fwd_smem_bytes<QR, NST, NW>();
    if (smem > 48 * 1024) {
        static bool done = false;
        if (!done) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (e != cudaSuccess) return e;
            done = true;
        }
    }
    k<<<grid, NW * 32, smem, s>>>(box, row, p);
    return cudaGetLastError();
}

// the compiled forward configurations (quad rows per stage, stages, warps)
#define DWT2_FWD_CFG_LIST(X) X(0, 2, 4, 4) X(1, 3, 3, 4) X(2, 1, 8, 4)

template <class Pipe, class OutT>
int launch_fwd_cfgs(const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p, int grid,
                    const FwdCfg& c, cudaStream_t s) {
#define DWT2_X(I_, QR_, NST_, NW_)                      \
    if (c.qr == QR_ && c.nst == NST_ && c.nw == NW_) \
        return launch_fwd_one<Pipe, OutT, QR_, NST_, NW_>(box, row, p, grid, s);
    DWT2_FWD_CFG_LIST(DWT2_X)
#undef DWT2_X
    return cudaErrorInvalidValue;
}

template <class OutT>
int launch_forward_t(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p,
                     int grid, const FwdCfg& c, cudaStream_t s) {
    if constexpr (std::is_same<OutT, int>::value) {
        if (wav != WAV_CDF53I) return cudaErrorInvalidValue;
        if (scheme == SCHEME_SEP) return launch_fwd_cfgs<Fwd53<SCHEME_SEP>, int>(box, row, p, grid, c, s);
        if (scheme == SCHEME_NONSEP) return launch_fwd_cfgs<Fwd53<SCHEME_NONSEP>, int>(box, row, p, grid, c, s);
        return cudaErrorInvalidValue;
    } else {
        if (wav != WAV_CDF97) return cudaErrorInvalidValue;
        if (scheme == SCHEME_NONSEP) return launch_fwd_cfgs<Fwd97<SCHEME_NONSEP>, OutT>(box, row, p, grid, c, s);
        if (scheme == SCHEME_REDUCED) return launch_fwd_cfgs<Fwd97<SCHEME_REDUCED>, OutT>(box, row, p, grid, c, s);
        if (scheme == SCHEME_SEP) return launch_fwd_cfgs<Fwd97<SCHEME_SEP>, OutT>(box, row, p, grid, c, s);
        return cudaErrorInvalidValue;
    }
}

template <class Pipe, class BT, bool ADJ>
int launch_inv_one(const InvParams& p, int grid, cudaStream_t s) {
    inv_kernel<Pipe, BT, ADJ, INV_NW><<<grid, INV_NW * 32, 0, s>>>(p);
    return cudaGetLastError();
}

template <class BT>
int launch_inverse_t(int wav, int scheme, const InvParams& p, int grid, cudaStream_t s) {
    if constexpr (std::is_same<BT, int>::value) {
        if (wav != WAV_CDF53I) return cudaErrorInvalidValue;
        if (scheme == SCHEME_SEP) return launch_inv_one<Inv53<SCHEME_SEP>, int, false>(p, grid, s);
        if (scheme == SCHEME_NONSEP) return launch_inv_one<Inv53<SCHEME_NONSEP>, int, false>(p, grid, s);
        return cudaErrorInvalidValue;
    } else {
        if (wav != WAV_CDF97) return cudaErrorInvalidValue;
        if (scheme == SCHEME_NONSEP) return launch_inv_one<Inv97<SCHEME_NONSEP>, BT, false>(p, grid, s);
        if (scheme == SCHEME_REDUCED) return launch_inv_one<Inv97<SCHEME_REDUCED>, BT, false>(p, grid, s);
        if (scheme == SCHEME_SEP) return launch_inv_one<Inv97<SCHEME_SEP>, BT, false>(p, grid, s);
        return cudaErrorInvalidValue;
    }
}

}  // namespace dwt2
