// band.cu -- row bands of one image: the partition of an image's rows into
// bands that transform independently (each on its own GPU, or one after the
// other on one), and the kernel that copies the rows a band owns from its own
// Mallat layout into the whole image's.
//
// A band owns input rows [own0, own1); both are multiples of 2^L (the last
// band ends at h), so the band's quads coincide with the image's quads at
// every level.  A level-L coefficient of quad row i depends on the input rows
// [2^L i - a(2^L - 1), 2^L (i + 1) - 1 + a(2^L - 1)], where a is the reach of
// one level in rows of its input (the half length of the longer analysis
// filter: 4 for CDF 9/7, 2 for CDF 5/3, 6 for DD 13/7).  A band therefore
// transforms rows [in0, in1) = [own0 - H, own1 + H) clipped to the image,
// with H = a(2^L - 1) rounded up to a multiple of 2^L: every coefficient it
// owns has its whole dependency cone inside real image rows, so it equals the
// coefficient of the whole-image transform computed with the same arithmetic,
// and the mirrored rows at the band's cut edges only reach coefficients that
// other bands own.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dwt2.h"
#include "internal.h"

namespace {

int reach_rows(int wavelet) {
    switch (wavelet) {
        case DWT2_CDF97: return 4;
        case DWT2_CDF53_INT: return 2;
        case DWT2_DD137: return 6;
        default: return -1;
    }
}

// own / in rows of one band; DWT2_OK or an error code
int band_rows(int wavelet, int levels, int h, int n_bands, int band, int32_t r[4]) {
    const int a = reach_rows(wavelet);
    if (a < 0 || levels < 1 || levels > 24 || h < 1 || n_bands < 1 || band < 0 || band >= n_bands)
        return DWT2_ERR_INVALID_ARG;
    const int64_t q = int64_t(1) << levels;
    // band boundaries: the multiples of 2^L nearest to r*h/n_bands
    auto cut = [&](int k) -> int64_t {
        if (k <= 0) return 0;
        if (k >= n_bands) return h;
        const int64_t t = (int64_t(2) * k * h + n_bands) / (2 * int64_t(n_bands));  // round(k h / n)
        return (t + q / 2) / q * q;
    };
    const int64_t o0 = cut(band), o1 = cut(band + 1);
    // every band must own at least one full quad row of the coarsest level
    for (int k = 0; k < n_bands; ++k)
        if (cut(k + 1) - cut(k) < q) return DWT2_ERR_INVALID_ARG;
    const int64_t halo = (int64_t(a) * (q - 1) + q - 1) / q * q;
    r[0] = int32_t(o0);
    r[1] = int32_t(o1);
    r[2] = int32_t(o0 - halo < 0 ? 0 : o0 - halo);
    r[3] = int32_t(o1 + halo > h ? h : o1 + halo);
    return DWT2_OK;
}

// One rectangle of the copy: rows [src_row, src_row + rows) of the band's
// coefficients go to rows [dst_row, ...) of the image's, columns
// [col0, col0 + cols) in both.
struct Rect {
    int32_t src_row, dst_row, rows, col0, cols;
};

int band_rects(int wavelet, int levels, int h, int w, int n_bands, int band, Rect* out, int max_rects) {
    int32_t r[4];
    const int rc = band_rows(wavelet, levels, h, n_bands, band, r);
    if (rc != DWT2_OK) return rc;
    if (w < 1) return DWT2_ERR_INVALID_ARG;
    const int64_t own0 = r[0], own1 = r[1], in0 = r[2], in1 = r[3];
    const bool last = own1 == h;
    int n = 0;
    auto add = [&](int64_t sr, int64_t dr, int64_t rows, int64_t c0, int64_t cols) {
        if (rows <= 0 || cols <= 0) return true;
        if (out) {  // without an output array the rectangles are only counted
            if (n >= max_rects) return false;
            out[n] = Rect{int32_t(sr), int32_t(dr), int32_t(rows), int32_t(c0), int32_t(cols)};
        }
        ++n;
        return true;
    };
    int64_t H = h, W = w, HL = in1 - in0;  // level input sizes: whole image, band
    for (int k = 1; k <= levels; ++k) {
        const int64_t hq = (H + 1) / 2, wq = (W + 1) / 2, hh = H / 2;
        const int64_t hql = (HL + 1) / 2;
        const int64_t o0 = own0 >> k, o1 = last ? hq : (own1 >> k), i0 = in0 >> k;
        // HL (and, at the last level, LL beside it): rows [o0, o1) of the top half
        if (!add(o0 - i0, o0, o1 - o0, wq, W - wq)) return DWT2_ERR_INVALID_ARG;
        // LH and HH: rows [o0, min(o1, hh)) of the bottom half, full width
        const int64_t e1 = o1 < hh ? o1 : hh;
        if (!add(hql + o0 - i0, hq + o0, e1 - o0, 0, W)) return DWT2_ERR_INVALID_ARG;
        if (k == levels && !add(o0 - i0, o0, o1 - o0, 0, wq)) return DWT2_ERR_INVALID_ARG;
        H = hq, W = wq, HL = hql;
    }
    return n;
}

constexpr int STITCH_MAX_RECTS = 3 * 24 + 1;
struct StitchLaunch {
    Rect rect[STITCH_MAX_RECTS];
    int n_rects;
    const char* src;
    char* dst;
    int64_t src_pitch, dst_pitch;  // elements
    int esize;                     // bytes per element
};

// One block row per (rectangle, row); threads stride over the columns.
__global__ void band_stitch_kernel(const __grid_constant__ StitchLaunch L) {
    for (int i = blockIdx.y; i < L.n_rects; i += gridDim.y) {
        const Rect& r = L.rect[i];
        for (int y = blockIdx.x; y < r.rows; y += gridDim.x) {
            const char* s = L.src + (int64_t(r.src_row + y) * L.src_pitch + r.col0) * L.esize;
            char* d = L.dst + (int64_t(r.dst_row + y) * L.dst_pitch + r.col0) * L.esize;
            if (L.esize == 4) {
                const uint32_t* s4 = reinterpret_cast<const uint32_t*>(s);
                uint32_t* d4 = reinterpret_cast<uint32_t*>(d);
                for (int x = threadIdx.x; x < r.cols; x += blockDim.x) d4[x] = s4[x];
            } else {
                const uint16_t* s2 = reinterpret_cast<const uint16_t*>(s);
                uint16_t* d2 = reinterpret_cast<uint16_t*>(d);
                for (int x = threadIdx.x; x < r.cols; x += blockDim.x) d2[x] = s2[x];
            }
        }
    }
}

}  // namespace

extern "C" {

int dwt2_band_rows(int wavelet, int levels, int h, int n_bands, int band, int32_t rows[4]) {
    if (!rows) return DWT2_ERR_INVALID_ARG;
    return band_rows(wavelet, levels, h, n_bands, band, rows);
}

int dwt2_band_rects(int wavelet, int levels, int h, int w, int n_bands, int band, int32_t* rects,
                    int max_rects) {
    if (max_rects < 0 || (max_rects > 0 && !rects)) return DWT2_ERR_INVALID_ARG;
    static_assert(sizeof(Rect) == 5 * sizeof(int32_t), "five int32 per rectangle");
    return band_rects(wavelet, levels, h, w, n_bands, band, reinterpret_cast<Rect*>(rects), max_rects);
}

int dwt2_band_stitch(int wavelet, int levels, int coef_dtype, int h, int w, int n_bands, int band,
                     const void* band_coef, int64_t band_pitch, void* coef, int64_t pitch, void* stream) {
    if (!band_coef || !coef || coef_dtype < DWT2_F32 || coef_dtype > DWT2_I32 || pitch < w || band_pitch < w)
        return DWT2_ERR_INVALID_ARG;
    StitchLaunch L;
    const int n = band_rects(wavelet, levels, h, w, n_bands, band, L.rect, STITCH_MAX_RECTS);
    if (n < 0) return n;
    L.n_rects = n;
    L.src = static_cast<const char*>(band_coef);
    L.dst = static_cast<char*>(coef);
    L.src_pitch = band_pitch;
    L.dst_pitch = pitch;
    L.esize = (coef_dtype == DWT2_F16 || coef_dtype == DWT2_BF16) ? 2 : 4;
    if (reinterpret_cast<uintptr_t>(band_coef) % L.esize || reinterpret_cast<uintptr_t>(coef) % L.esize)
        return DWT2_ERR_MISALIGNED;
    int32_t r[4];
    band_rows(wavelet, levels, h, n_bands, band, r);
    const int rows_max = (r[1] - r[0] + 1) / 2 + 1;
    dim3 grid(unsigned(rows_max < 4096 ? rows_max : 4096), unsigned(n));
    band_stitch_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(L);
    return cudaGetLastError() == cudaSuccess ? DWT2_OK : DWT2_ERR_CUDA;
}

}  // extern "C"
