// kernels.cuh -- the transform kernels of one pyramid level.
//
// Work decomposition: the level is cut into vertical strips of 60 output
// quads (120 pixels; a warp loads 128 pixels, 4 on each side are halo) and
// horizontal segments of seg_rows output quad rows.  One (strip, segment)
// pair is a unit of work for one warp.  A warp streams the quad rows of its
// unit top to bottom through the row pipeline of the scheme (schemes.cuh),
// starting two quad rows above the segment (warm-up) and running LAG rows
// past it.
//
// Forward: each warp owns a ring of NST shared-memory stages of QR quad rows
// (2*QR pixel rows x 128 pixels) filled by 2-D TMA loads that complete on one
// mbarrier per stage; lane 0 refills a stage once the warp has read it.  Rows
// outside the image are fetched from their whole-sample mirror rows (one
// single-row TMA box per pixel row); columns outside the image are mirrored in
// shared memory by the edge strips.  With the symmetric extension in place the
// lifting needs no boundary cases: every step preserves the symmetry, so the
// exact per-step mirrored result appears inside the image.
//
// Inverse and adjoint: the four bands are read with vector loads, two quad
// rows ahead of the pipeline.  The inverse reads mirrored band positions at the
// edges (the extension of the coefficients that the symmetric image extension
// produces); the adjoint reads zeros there and applies the transposed boundary
// weights of Adj97 instead.
#pragma once

#include "schemes.cuh"

namespace dwt2 {

template <class CT>
__device__ __forceinline__ void ld4_smem(const CT* p, CT (&v)[4]);
template <>
__device__ __forceinline__ void ld4_smem<float>(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
template <>
__device__ __forceinline__ void ld4_smem<int>(const int* p, int (&v)[4]) {
    const int4 t = *reinterpret_cast<const int4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}

template <class CT>
__device__ __forceinline__ void st4(CT* p, CT a, CT b, CT c, CT d);
template <>
__device__ __forceinline__ void st4<float>(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ void st4<int>(int* p, int a, int b, int c, int d) {
    *reinterpret_cast<int4*>(p) = make_int4(a, b, c, d);
}

// shared-memory bytes of a forward launch
template <int QR, int NST, int NW>
constexpr size_t fwd_smem_bytes() {
    return size_t(NW) * NST * (2 * QR * STRIP_PX * 4) + size_t(NW) * NST * 8;
}

// ------------------------------------------------------------------ forward
template <class Pipe, class OutT, int QR, int NST, int NW>
__global__ void __launch_bounds__(NW * 32)
    fwd_tma_kernel(const __grid_constant__ CUtensorMap tm_box, const __grid_constant__ CUtensorMap tm_row,
                   const FwdParams p) {
    using CT = typename Pipe::CT;
    constexpr int ROWS = 2 * QR;
    constexpr int STAGE_ELEMS = ROWS * STRIP_PX;
    constexpr unsigned STAGE_BYTES = STAGE_ELEMS * 4u;
    extern __shared__ __align__(128) unsigned char smem[];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CT* bufs = reinterpret_cast<CT*>(smem) + warp * NST * STAGE_ELEMS;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(NW) * NST * STAGE_BYTES) + warp * NST;

    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NST; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
        tma_prefetch_desc(&tm_box);
        tma_prefetch_desc(&tm_row);
    }
    __syncwarp();

    uint32_t gstage = 0;  // stages consumed by this warp so far (slot / phase)
    for (int unit = blockIdx.x * NW + warp; unit < p.n_units; unit += gridDim.x * NW) {
        const int s = unit % p.n_strips, g = unit / p.n_strips;
        const int R0 = g * p.seg_rows;
        const int R1 = min(R0 + p.seg_rows, p.hq);
        const int A0 = R0 - 2;                           // first quad row streamed
        const int n_arr = (R1 - R0) + 2 + Pipe::LAG;     // quad rows streamed
        const int NT = (n_arr + QR - 1) / QR;            // stages
        const int x0 = s * (2 * OUT_Q) - 2 * HALO_Q;     // first pixel column (multiple of 4)
        const int jb = x0 / 2 + 2 * lane;                // first quad column of this lane
        const bool edge = (x0 < 0) || (x0 + STRIP_PX > p.w);

        auto issue = [&](int t, int slot) {
            const int y0 = 2 * (A0 + t * QR);
            CT* dst = bufs + slot * STAGE_ELEMS;
            mbar_expect_tx(&bars[slot], STAGE_BYTES);
            if (y0 >= 0 && y0 + ROWS <= p.h) {
                tma_load_2d(dst, &tm_box, x0, y0, &bars[slot]);
            } else {
#pragma unroll 1
                for (int r = 0; r < ROWS; ++r)
                    tma_load_2d(dst + r * STRIP_PX, &tm_row, x0, fold_ws(y0 + r, p.h), &bars[slot]);
            }
        };

        if (lane == 0) {
            for (int t = 0; t < NST && t < NT; ++t) issue(t, (gstage + t) % NST);
        }

        Pipe pipe;
        pipe.init();
        bool ok = true;
        for (int t = 0; t < NT; ++t) {
            const uint32_t gs = gstage + t;
            const int slot = gs % NST;
            if (!mbar_wait_bounded(&bars[slot], (gs / NST) & 1u, p.status, p.timeout_ns)) {
                // give the copies still in flight a bounded time to land
                for (int u = t + 1; u < NT && u < t + NST; ++u) {
                    const uint32_t gu = gstage + u;
                    mbar_wait_bounded(&bars[gu % NST], (gu / NST) & 1u, nullptr, p.timeout_ns);
                }
                ok = false;
                break;
            }
            const CT* stage = bufs + slot * STAGE_ELEMS;
#pragma unroll
            for (int qr = 0; qr < QR; ++qr) {
                const int vi = A0 + t * QR + qr;  // quad row streamed now
                const CT* s0 = stage + (2 * qr) * STRIP_PX;
                const CT* s1 = s0 + STRIP_PX;
                CT e[4], o[4];
                ld4_smem<CT>(s0 + 4 * lane, e);
                ld4_smem<CT>(s1 + 4 * lane, o);
                if (edge) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int px = x0 + 4 * lane + k;
                        if (px < 0 || px >= p.w) {
                            const int src = fold_ws(px, p.w) - x0;
                            const bool in = (src >= 0) && (src < STRIP_PX);
                            e[k] = in ? s0[src] : CT(0);
                            o[k] = in ? s1[src] : CT(0);
                        }
                    }
                }
                Row<CT> in;
                in.c1[0] = e[0], in.c2[0] = e[1], in.c1[1] = e[2], in.c2[1] = e[3];
                in.c3[0] = o[0], in.c4[0] = o[1], in.c3[1] = o[2], in.c4[1] = o[3];
                const Row<CT> out = pipe.arrive(in, vi);
                const int oi = vi - Pipe::LAG;
                if (oi >= R0 && oi < R1) {
                    const bool lo = (lane >= 1) && (lane <= 30);
                    const bool e0 = lo && jb < p.wq, e1 = lo && jb + 1 < p.wq;
                    const bool d0 = lo && jb < p.wh, d1 = lo && jb + 1 < p.wh;
                    const bool odd_row = oi < p.hh;
                    OutT* crow = reinterpret_cast<OutT*>(p.coef) + int64_t(oi) * p.coef_pitch;
                    OutT* crow_b = reinterpret_cast<OutT*>(p.coef) + int64_t(p.hq + oi) * p.coef_pitch;
                    if (p.ll_is_ct) {
                        CT* lrow = reinterpret_cast<CT*>(p.ll) + int64_t(oi) * p.ll_pitch;
                        store_pair<CT, CT>(lrow, jb, out.c1[0], out.c1[1], e0, e1, p.vec_ll);
                    } else {
                        OutT* lrow = reinterpret_cast<OutT*>(p.ll) + int64_t(oi) * p.ll_pitch;
                        store_pair<OutT, CT>(lrow, jb, out.c1[0], out.c1[1], e0, e1, p.vec_ll);
                    }
                    store_pair<OutT, CT>(crow + p.wq, jb, out.c2[0], out.c2[1], d0, d1, p.vec_hi);
                    if (odd_row) {
                        store_pair<OutT, CT>(crow_b, jb, out.c3[0], out.c3[1], e0, e1, p.vec_lo);
                        store_pair<OutT, CT>(crow_b + p.wq, jb, out.c4[0], out.c4[1], d0, d1, p.vec_hi);
                    }
                }
            }
            __syncwarp();
            if (lane == 0 && t + NST < NT) issue(t + NST, slot);
        }
        if (!ok) return;
        gstage += NT;
    }
}

// ------------------------------------------------- band loads (inverse, adjoint)
template <class T>
__device__ __forceinline__ void ld_pair(const T* p, float& a, float& b, bool vec) {
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            const float2 t = *reinterpret_cast<const float2*>(p);
            a = t.x, b = t.y;
        } else if constexpr (std::is_same<T, __half>::value) {
            const __half2 t = *reinterpret_cast<const __half2*>(p);
            a = __low2float(t), b = __high2float(t);
        } else {
            const __nv_bfloat162 t = *reinterpret_cast<const __nv_bfloat162*>(p);
            a = __low2float(t), b = __high2float(t);
        }
    } else {
        a = Cvt<T>::from(p[0]);
        b = Cvt<T>::from(p[1]);
    }
}
__device__ __forceinline__ void ld_pair(const int* p, int& a, int& b, bool vec) {
    if (vec) {
        const int2 t = *reinterpret_cast<const int2*>(p);
        a = t.x, b = t.y;
    } else {
        a = p[0];
        b = p[1];
    }
}

template <class T, class CT>
__device__ __forceinline__ CT ld_one(const T* p) {
    return CT(Cvt<T>::from(*p));
}

// One quad row of the lane's two quads from the four bands.  MIRROR: positions
// outside the image read their mirror images; otherwise they read zero.
template <class CT, class BT, bool MIRROR>
__device__ __forceinline__ Row<CT> load_bands(const InvParams& p, int vi, int jb, bool fast) {
    Row<CT> r;
    const BT* coef = reinterpret_cast<const BT*>(p.coef);
    if (fast) {  // whole strip and row inside the bands: direct pair loads
        const int64_t re = vi, ro = vi;
        const BT* hl = coef + re * p.coef_pitch + p.wq;
        const BT* lh = coef + (p.hq + ro) * p.coef_pitch;
        const BT* hh = lh + p.wq;
        if (p.ll_is_ct) {
            const CT* ll = reinterpret_cast<const CT*>(p.ll) + re * p.ll_pitch;
            ld_pair(ll + jb, r.c1[0], r.c1[1], p.vec_ll);
        } else {
            const BT* ll = reinterpret_cast<const BT*>(p.ll) + re * p.ll_pitch;
            ld_pair(ll + jb, r.c1[0], r.c1[1], p.vec_ll);
        }
        ld_pair(hl + jb, r.c2[0], r.c2[1], p.vec_in_hi);
        ld_pair(lh + jb, r.c3[0], r.c3[1], p.vec_in_lo);
        ld_pair(hh + jb, r.c4[0], r.c4[1], p.vec_in_hi);
        return r;
    }
    int re, ro;
    bool rev, rov;
    if (MIRROR) {
        re = fold_ws(2 * vi, p.h) >> 1;
        ro = fold_ws(2 * vi + 1, p.h) >> 1;
        rev = rov = true;
    } else {
        rev = (vi >= 0) && (vi < p.hq);
        rov = (vi >= 0) && (vi < p.hh);
        re = rev ? vi : 0;
        ro = rov ? vi : 0;
    }
    // defensive clamps keep every address inside the bands
    re = min(max(re, 0), p.hq - 1);
    ro = min(max(ro, 0), max(p.hh - 1, 0));
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int j = jb + q;
        int ce, co;
        bool cev, cov;
        if (MIRROR) {
            ce = fold_ws(2 * j, p.w) >> 1;
            co = fold_ws(2 * j + 1, p.w) >> 1;
            cev = cov = true;
        } else {
            cev = (j >= 0) && (j < p.wq);
            cov = (j >= 0) && (j < p.wh);
            ce = cev ? j : 0;
            co = cov ? j : 0;
        }
        ce = min(max(ce, 0), p.wq - 1);
        co = min(max(co, 0), max(p.wh - 1, 0));
        CT v1, v2, v3, v4;
        if (p.ll_is_ct)
            v1 = reinterpret_cast<const CT*>(p.ll)[int64_t(re) * p.ll_pitch + ce];
        else
            v1 = ld_one<BT, CT>(reinterpret_cast<const BT*>(p.ll) + int64_t(re) * p.ll_pitch + ce);
        v2 = ld_one<BT, CT>(coef + int64_t(re) * p.coef_pitch + p.wq + co);
        v3 = ld_one<BT, CT>(coef + int64_t(p.hq + ro) * p.coef_pitch + ce);
        v4 = ld_one<BT, CT>(coef + int64_t(p.hq + ro) * p.coef_pitch + p.wq + co);
        r.c1[q] = (rev && cev) ? v1 : CT(0);
        r.c2[q] = (rev && cov) ? v2 : CT(0);
        r.c3[q] = (rov && cev) ? v3 : CT(0);
        r.c4[q] = (rov && cov) ? v4 : CT(0);
    }
    return r;
}

// --------------------------------------------------------- inverse / adjoint
// Pipe: Inv97<S>, Inv53<S> or Adj97.  BT: coefficient element type.
template <class Pipe, class BT, bool ADJ, int NW>
__global__ void __launch_bounds__(NW * 32) inv_kernel(const InvParams p) {
    using CT = typename Pipe::CT;
    constexpr bool MIRROR = !ADJ;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int unit = blockIdx.x * NW + warp; unit < p.n_units; unit += gridDim.x * NW) {
        const int s = unit % p.n_strips, g = unit / p.n_strips;
        const int R0 = g * p.seg_rows;
        const int R1 = min(R0 + p.seg_rows, p.hq);
        const int A0 = R0 - 2;
        const int n_arr = (R1 - R0) + 2 + Pipe::LAG;
        const int x0 = s * (2 * OUT_Q) - 2 * HALO_Q;
        const int jb = x0 / 2 + 2 * lane;
        // the whole strip reads only existing band columns
        const bool fast_cols = (x0 >= 0) && (x0 / 2 + 2 * 32 <= p.wh);

        Pipe pipe;
        pipe.init();
        if constexpr (ADJ) {
#pragma unroll
            for (int q = 0; q < QL; ++q) pipe.hw[q] = axis_weights(jb + q, p.w);
            pipe.h = p.h;
        }
        auto fast_row = [&](int vi) { return fast_cols && vi >= 0 && 2 * vi + 1 < p.h; };

        Row<CT> n1 = load_bands<CT, BT, MIRROR>(p, A0, jb, fast_row(A0));
        Row<CT> n2 = load_bands<CT, BT, MIRROR>(p, A0 + 1, jb, fast_row(A0 + 1));
        for (int a = 0; a < n_arr; ++a) {
            const int vi = A0 + a;
            const Row<CT> cur = n1;
            n1 = n2;
            if (a + 2 < n_arr) n2 = load_bands<CT, BT, MIRROR>(p, vi + 2, jb, fast_row(vi + 2));
            const Row<CT> out = pipe.arrive(cur, vi);
            const int oi = vi - Pipe::LAG;
            if (oi < R0 || oi >= R1) continue;
            const bool lo = (lane >= 1) && (lane <= 30);
            const int px = 2 * jb;  // first pixel column of the lane
            CT* row_e = reinterpret_cast<CT*>(p.out) + int64_t(2 * oi) * p.out_pitch;
            CT* row_o = row_e + p.out_pitch;
            const bool has_o = 2 * oi + 1 < p.h;
            if (lo && p.vec_out && px + 3 < p.w) {
                st4<CT>(row_e + px, out.c1[0], out.c2[0], out.c1[1], out.c2[1]);
                if (has_o) st4<CT>(row_o + px, out.c3[0], out.c4[0], out.c3[1], out.c4[1]);
            } else if (lo) {
                const CT ev[4] = {out.c1[0], out.c2[0], out.c1[1], out.c2[1]};
                const CT od[4] = {out.c3[0], out.c4[0], out.c3[1], out.c4[1]};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (px + k < p.w) {
                        row_e[px + k] = ev[k];
                        if (has_o) row_o[px + k] = od[k];
                    }
                }
            }
        }
    }
}

}  // namespace dwt2
