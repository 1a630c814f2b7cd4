// schemes.cuh -- the lifting steps of every scheme, applied to one quad row of
// one lane, and the row pipelines that stream quad rows through them.
//
// Notation (Barina et al., arXiv:1704.08657, Background and Proposed
// Schemes): a quad is (c1, c2, c3, c4) = (x[2i][2j], x[2i][2j+1],
// x[2i+1][2j], x[2i+1][2j+1]).  P acts horizontally, P* vertically.
// Predict P = a(1 + z) reads the quad itself and the quad to the right (or
// below for P*); update U = b(1 + z^-1) reads the quad itself and the quad to
// the left (or above).
//
//   spatial predict T_P:  c2 += P c1;  c3 += P* c1;  c4 += PP* c1 + P* c2 + P c3
//   spatial update  S_U:  c1 += U c2 + U* c3 + UU* c4;  c2 += U* c4;  c3 += U c4
//
// with all operands taken before the step.  Quad rows stream top to bottom
// through the registers of a lane (QL quads per lane): a step that reads the
// row below runs one row later than the step before it; a step that reads the
// row above takes that row's pre-step values from a carry saved when the step
// ran on it.  Horizontal neighbours come from the next / previous lane by
// shuffle.
//
// Pipelines are driven by a compile-time phase PH (the arrival index modulo
// 6): the rows rotate through a ring of LAG+1 slots and the carries through
// two slots, so that a group of 6 unrolled arrivals needs no register copies.
#pragma once

#include <type_traits>

#include "dev_common.cuh"

namespace dwt2 {

// CDF 9/7 lifting constants (alpha, beta, gamma, delta) and scaling zeta.
struct C97 {
    static constexpr double Ad = -1.586134342, Bd = -0.052980119, Gd = 0.882911076, Dd = 0.443506852,
                            Zd = 1.149604398;
    static constexpr float A = float(Ad), B = float(Bd), G = float(Gd), D = float(Dd);
    static constexpr float AA = float(Ad * Ad), BB = float(Bd * Bd), GG = float(Gd * Gd), DD = float(Dd * Dd);
    static constexpr float ZZ = float(Zd * Zd), IZZ = float(1.0 / (Zd * Zd));
};

constexpr int PHASES = 6;  // arrivals per unrolled group

template <class CT, int QL>
struct Row {
    CT c1[QL], c2[QL], c3[QL], c4[QL];
};

// Strip and segment geometry of a pipeline: halo quads on each side of a
// strip (a finished quad depends on input quads up to that far minus one; an
// even count keeps a strip's first pixel a multiple of four) and warm-up quad
// rows streamed above a segment.  Pipelines that declare neither use two and
// two.
template <class Pipe, class = void>
struct PipeGeom {
    static constexpr int HALO = 2, WARM = 2;
};
template <class Pipe>
struct PipeGeom<Pipe, std::void_t<decltype(Pipe::HALO)>> {
    static constexpr int HALO = Pipe::HALO, WARM = Pipe::WARM;
};

template <class CT, int QL>
__device__ __forceinline__ void zero_row(Row<CT, QL>& r) {
#pragma unroll
    for (int q = 0; q < QL; ++q) r.c1[q] = r.c2[q] = r.c3[q] = r.c4[q] = CT(0);
}

// values of the quad to the right / left of each of the lane's quads
template <class CT, int QL>
__device__ __forceinline__ void right_of(const CT (&x)[QL], CT (&r)[QL]) {
    const CT nxt = __shfl_down_sync(FULL, x[0], 1);
#pragma unroll
    for (int q = 0; q + 1 < QL; ++q) r[q] = x[q + 1];
    r[QL - 1] = nxt;
}

template <class CT, int QL>
__device__ __forceinline__ void left_of(const CT (&x)[QL], CT (&l)[QL]) {
    const CT prv = __shfl_up_sync(FULL, x[QL - 1], 1);
    l[0] = prv;
#pragma unroll
    for (int q = 1; q < QL; ++q) l[q] = x[q - 1];
}

// carries of an update step: the row above, before the step
template <int QL>
struct Carry3 {
    float c3[QL], c4[QL], l4[QL];  // c3, c4 and the c4 of the quad to the left
};
template <class CT, int QL>
struct Carry2 {
    CT c3[QL], c4[QL];
};

template <int QL>
__device__ __forceinline__ void zero_carry(Carry3<QL>& c) {
#pragma unroll
    for (int q = 0; q < QL; ++q) c.c3[q] = c.c4[q] = c.l4[q] = 0.f;
}
template <class CT, int QL>
__device__ __forceinline__ void zero_carry(Carry2<CT, QL>& c) {
#pragma unroll
    for (int q = 0; q < QL; ++q) c.c3[q] = c.c4[q] = CT(0);
}

// ============================================================ CDF 9/7 float

// --- non-separable lifting (Proposed Schemes) ------------------------------
// T_P on row X with the row below D, P = a(1 + z): every operand pre-step.
template <int QL>
__device__ __forceinline__ void ns_predict(Row<float, QL>& X, const Row<float, QL>& D, float a, float aa) {
    float r1[QL], r3[QL], dr1[QL];
    right_of(X.c1, r1);
    right_of(X.c3, r3);
    right_of(D.c1, dr1);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const float s1 = X.c1[q] + r1[q];                         // P c1
        const float sd = D.c1[q] + dr1[q];                        // P c1 of the row below
        const float t = (X.c3[q] + r3[q]) + (X.c2[q] + D.c2[q]);  // P c3 + P* c2
        const float c4 = fmaf(a, t, X.c4[q]);
        X.c4[q] = fmaf(aa, s1 + sd, c4);                          // + PP* c1
        X.c2[q] = fmaf(a, s1, X.c2[q]);
        X.c3[q] = fmaf(a, X.c1[q] + D.c1[q], X.c3[q]);            // P* c1
    }
}

// S_U on row X with the carry C of the row above, U = b(1 + z^-1); the
// row's own pre-step values become the carry N for the row below.
template <int QL>
__device__ __forceinline__ void ns_update(Row<float, QL>& X, const Carry3<QL>& C, Carry3<QL>& N, float b,
                                          float bb) {
    float l2[QL], l4[QL];
    left_of(X.c2, l2);
    left_of(X.c4, l4);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        N.c3[q] = X.c3[q];
        N.c4[q] = X.c4[q];
        N.l4[q] = l4[q];
        const float h = l2[q] + X.c2[q];                              // U c2
        const float v = C.c3[q] + X.c3[q];                            // U* c3
        const float dg = (C.l4[q] + C.c4[q]) + (l4[q] + X.c4[q]);     // UU* c4
        X.c1[q] = fmaf(b, h + v, fmaf(bb, dg, X.c1[q]));
        X.c2[q] = fmaf(b, C.c4[q] + X.c4[q], X.c2[q]);                // U* c4
        X.c3[q] = fmaf(b, l4[q] + X.c4[q], X.c3[q]);                  // U c4
    }
}

// --- reduced operations (Optimization Approach) -----------------------------
// P = P0 + P1 with P0 = a (own quad) and P1 = a z (neighbour).  T_{P1} first,
// on pre-step values, then T_{P0}^H and T_{P0}^V inside the quad.
template <int QL>
__device__ __forceinline__ void rd_predict(Row<float, QL>& X, const Row<float, QL>& D, float a, float aa) {
    float r1[QL], r3[QL], dr1[QL];
    right_of(X.c1, r1);
    right_of(X.c3, r3);
    right_of(D.c1, dr1);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        float c2 = fmaf(a, r1[q], X.c2[q]);       // P1 c1
        float c3 = fmaf(a, D.c1[q], X.c3[q]);     // P1* c1
        float c4 = fmaf(a, r3[q], X.c4[q]);       // P1 c3
        c4 = fmaf(a, D.c2[q], c4);                // P1* c2
        c4 = fmaf(aa, dr1[q], c4);                // P1 P1* c1
        c2 = fmaf(a, X.c1[q], c2);                // T_{P0}^H
        c4 = fmaf(a, c3, c4);
        c3 = fmaf(a, X.c1[q], c3);                // T_{P0}^V
        c4 = fmaf(a, c2, c4);
        X.c2[q] = c2;
        X.c3[q] = c3;
        X.c4[q] = c4;
    }
}

// U = U0 + U1 with U0 = b and U1 = b z^-1: S_{U1}, then S_{U0}^H, S_{U0}^V.
template <int QL>
__device__ __forceinline__ void rd_update(Row<float, QL>& X, const Carry3<QL>& C, Carry3<QL>& N, float b,
                                          float bb) {
    float l2[QL], l4[QL];
    left_of(X.c2, l2);
    left_of(X.c4, l4);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        N.c3[q] = X.c3[q];
        N.c4[q] = X.c4[q];
        N.l4[q] = l4[q];
        float c1 = fmaf(b, l2[q], X.c1[q]);       // U1 c2
        c1 = fmaf(b, C.c3[q], c1);                // U1* c3
        c1 = fmaf(bb, C.l4[q], c1);               // U1 U1* c4
        float c2 = fmaf(b, C.c4[q], X.c2[q]);     // U1* c4
        float c3 = fmaf(b, l4[q], X.c3[q]);       // U1 c4
        c1 = fmaf(b, c2, c1);                     // S_{U0}^H
        c3 = fmaf(b, X.c4[q], c3);
        c1 = fmaf(b, c3, c1);                     // S_{U0}^V
        c2 = fmaf(b, X.c4[q], c2);
        X.c1[q] = c1;
        X.c2[q] = c2;
        X.c3[q] = c3;
    }
}

// inverse of rd_update: undo S_{U0}^V, S_{U0}^H inside the quad, then S_{-U1}
// (its pre-step operands are the post-undo values of the neighbours).
template <int QL>
__device__ __forceinline__ void rdi_update(Row<float, QL>& X, const Carry3<QL>& C, Carry3<QL>& N, float b,
                                           float bb) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c1[q] = fmaf(-b, X.c3[q], X.c1[q]);
        X.c2[q] = fmaf(-b, X.c4[q], X.c2[q]);
        X.c1[q] = fmaf(-b, X.c2[q], X.c1[q]);
        X.c3[q] = fmaf(-b, X.c4[q], X.c3[q]);
    }
    float l2[QL], l4[QL];
    left_of(X.c2, l2);
    left_of(X.c4, l4);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        N.c3[q] = X.c3[q];
        N.c4[q] = X.c4[q];
        N.l4[q] = l4[q];
        float c1 = fmaf(-b, l2[q], X.c1[q]);
        c1 = fmaf(-b, C.c3[q], c1);
        X.c1[q] = fmaf(bb, C.l4[q], c1);
        X.c2[q] = fmaf(-b, C.c4[q], X.c2[q]);
        X.c3[q] = fmaf(-b, l4[q], X.c3[q]);
    }
}

// inverse of rd_predict, part 1 (inside the quad): undo T_{P0}^V, T_{P0}^H.
template <int QL>
__device__ __forceinline__ void rdi_predict_local(Row<float, QL>& X, float a) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c4[q] = fmaf(-a, X.c2[q], X.c4[q]);
        X.c3[q] = fmaf(-a, X.c1[q], X.c3[q]);
        X.c4[q] = fmaf(-a, X.c3[q], X.c4[q]);
        X.c2[q] = fmaf(-a, X.c1[q], X.c2[q]);
    }
}

// inverse of rd_predict, part 2: T_{-P1}; the row below must have had part 1.
template <int QL>
__device__ __forceinline__ void rdi_predict_exch(Row<float, QL>& X, const Row<float, QL>& D, float a, float aa) {
    float r1[QL], r3[QL], dr1[QL];
    right_of(X.c1, r1);
    right_of(X.c3, r3);
    right_of(D.c1, dr1);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        float c4 = fmaf(-a, r3[q], X.c4[q]);
        c4 = fmaf(-a, D.c2[q], c4);
        X.c4[q] = fmaf(aa, dr1[q], c4);
        X.c2[q] = fmaf(-a, r1[q], X.c2[q]);
        X.c3[q] = fmaf(-a, D.c1[q], X.c3[q]);
    }
}

// --- separable lifting (Background) -----------------------------------------
template <int QL>
__device__ __forceinline__ void sp_th(Row<float, QL>& X, float a) {  // T_P^H
    float r1[QL], r3[QL];
    right_of(X.c1, r1);
    right_of(X.c3, r3);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c2[q] = fmaf(a, X.c1[q] + r1[q], X.c2[q]);
        X.c4[q] = fmaf(a, X.c3[q] + r3[q], X.c4[q]);
    }
}
template <int QL>
__device__ __forceinline__ void sp_tv(Row<float, QL>& X, const Row<float, QL>& D, float a) {  // T_P^V
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c3[q] = fmaf(a, X.c1[q] + D.c1[q], X.c3[q]);
        X.c4[q] = fmaf(a, X.c2[q] + D.c2[q], X.c4[q]);
    }
}
template <int QL>
__device__ __forceinline__ void sp_sh(Row<float, QL>& X, float b) {  // S_U^H
    float l2[QL], l4[QL];
    left_of(X.c2, l2);
    left_of(X.c4, l4);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c1[q] = fmaf(b, l2[q] + X.c2[q], X.c1[q]);
        X.c3[q] = fmaf(b, l4[q] + X.c4[q], X.c3[q]);
    }
}
template <int QL>
__device__ __forceinline__ void sp_sv(Row<float, QL>& X, const Carry2<float, QL>& C, Carry2<float, QL>& N,
                                      float b) {  // S_U^V
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c1[q] = fmaf(b, C.c3[q] + X.c3[q], X.c1[q]);
        X.c2[q] = fmaf(b, C.c4[q] + X.c4[q], X.c2[q]);
        N.c3[q] = X.c3[q];
        N.c4[q] = X.c4[q];
    }
}

// scaling: per axis low * zeta, high / zeta
template <int QL>
__device__ __forceinline__ void scale97(Row<float, QL>& X) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c1[q] *= C97::ZZ;
        X.c4[q] *= C97::IZZ;
    }
}
template <int QL>
__device__ __forceinline__ void unscale97(Row<float, QL>& X) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c1[q] *= C97::IZZ;
        X.c4[q] *= C97::ZZ;
    }
}

// ---------------------------------------------------------- 9/7 pipelines
// slot<PH>() is where arrival PH's quad row is loaded; step<PH>(row) runs the
// steps due at that arrival and returns the finished row LAG rows above it.
template <int SCHEME, int QL>
struct Fwd97 {
    static constexpr int LAG = 2;
    using CT = float;
    using R = Row<float, QL>;
    R rw[3];
    Carry3<QL> ka[2], kb[2];
    Carry2<float, QL> sa[2], sb[2];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 3; ++i) zero_row(rw[i]);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            zero_carry(ka[i]);
            zero_carry(kb[i]);
            zero_carry(sa[i]);
            zero_carry(sb[i]);
        }
    }
    template <int PH>
    __device__ __forceinline__ R& slot() {
        return rw[PH % 3];
    }
    template <int PH>
    __device__ __forceinline__ R& step(int /*row*/) {
        R& r0 = rw[PH % 3];
        R& r1 = rw[(PH + 2) % 3];
        R& r2 = rw[(PH + 1) % 3];
        constexpr int c = PH & 1, n = c ^ 1;
        if constexpr (SCHEME == SCHEME_NONSEP) {
            ns_predict(r1, r0, C97::A, C97::AA);
            ns_update(r1, ka[c], ka[n], C97::B, C97::BB);
            ns_predict(r2, r1, C97::G, C97::GG);
            ns_update(r2, kb[c], kb[n], C97::D, C97::DD);
        } else if constexpr (SCHEME == SCHEME_REDUCED) {
            rd_predict(r1, r0, C97::A, C97::AA);
            rd_update(r1, ka[c], ka[n], C97::B, C97::BB);
            rd_predict(r2, r1, C97::G, C97::GG);
            rd_update(r2, kb[c], kb[n], C97::D, C97::DD);
        } else {
            sp_th(r0, C97::A);
            sp_tv(r1, r0, C97::A);
            sp_sh(r1, C97::B);
            sp_sv(r1, sa[c], sa[n], C97::B);
            sp_th(r1, C97::G);
            sp_tv(r2, r1, C97::G);
            sp_sh(r2, C97::D);
            sp_sv(r2, sb[c], sb[n], C97::D);
        }
        scale97(r2);
        return r2;
    }
};

// --- polyconvolution (Proposed Schemes, N_{P,U}) -----------------------------
// One lifting pair (P, U) as one step on pre-pair values: with V = 1 + PU the
// pair's 4x4 matrix is the tensor product of the vertical [V* U*; P* 1] and
// the horizontal [V U; P 1] 1-D pair matrices.  A row streams through the
// horizontal part (h = [V U; P 1] on (c1, c2) and on (c3, c4), one exchange
// of pre-pair neighbour values), and the vertical part combines the rows
// above, here and below of h from registers.  V is applied as the 3-tap
// filter 1 + ab(z^-1 + 2 + z) rather than as a predict followed by an update.
// In this row-streaming design the separable and non-separable polyconvolution
// schemes of the paper coincide: neither has a barrier between its
// horizontal and vertical parts.
template <int QL>
__device__ __forceinline__ void pc_horiz(Row<float, QL>& X, float a, float b, float ab, float k0) {
    float l1[QL], r1[QL], l2[QL], l3[QL], r3[QL], l4[QL];
    left_of(X.c1, l1);
    right_of(X.c1, r1);
    left_of(X.c2, l2);
    left_of(X.c3, l3);
    right_of(X.c3, r3);
    left_of(X.c4, l4);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const float h1 = fmaf(ab, l1[q] + r1[q], fmaf(b, l2[q] + X.c2[q], k0 * X.c1[q]));  // V c1 + U c2
        const float h2 = fmaf(a, X.c1[q] + r1[q], X.c2[q]);                                // P c1 + c2
        const float h3 = fmaf(ab, l3[q] + r3[q], fmaf(b, l4[q] + X.c4[q], k0 * X.c3[q]));  // V c3 + U c4
        const float h4 = fmaf(a, X.c3[q] + r3[q], X.c4[q]);                                // P c3 + c4
        X.c1[q] = h1;
        X.c2[q] = h2;
        X.c3[q] = h3;
        X.c4[q] = h4;
    }
}

// O = [V* U*; P* 1] on the columns (h1, h3) and (h2, h4) of the rows above
// (Up), here (H) and below (Dn).
template <int QL>
__device__ __forceinline__ void pc_vert(Row<float, QL>& O, const Row<float, QL>& Up, const Row<float, QL>& H,
                                        const Row<float, QL>& Dn, float a, float b, float ab, float k0) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        O.c1[q] = fmaf(ab, Up.c1[q] + Dn.c1[q], fmaf(b, Up.c3[q] + H.c3[q], k0 * H.c1[q]));  // V* h1 + U* h3
        O.c3[q] = fmaf(a, H.c1[q] + Dn.c1[q], H.c3[q]);                                      // P* h1 + h3
        O.c2[q] = fmaf(ab, Up.c2[q] + Dn.c2[q], fmaf(b, Up.c4[q] + H.c4[q], k0 * H.c2[q]));  // V* h2 + U* h4
        O.c4[q] = fmaf(a, H.c2[q] + Dn.c2[q], H.c4[q]);                                      // P* h2 + h4
    }
}

// CDF 9/7 by polyconvolution: pair (alpha, beta) on arrival n gives row n-1,
// pair (gamma, delta) then gives row n-2; each pair keeps three rows of h.
template <int QL>
struct Fwd97PC {
    static constexpr int LAG = 2;
    using CT = float;
    using R = Row<float, QL>;
    static constexpr float AB = float(C97::Ad * C97::Bd), K1 = float(1.0 + 2.0 * C97::Ad * C97::Bd);
    static constexpr float GD = float(C97::Gd * C97::Dd), K2 = float(1.0 + 2.0 * C97::Gd * C97::Dd);
    R w1[3], w2[3], o;
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            zero_row(w1[i]);
            zero_row(w2[i]);
        }
    }
    template <int PH>
    __device__ __forceinline__ R& slot() {
        return w1[PH % 3];
    }
    template <int PH>
    __device__ __forceinline__ R& step(int /*row*/) {
        R& x = w1[PH % 3];  // arrival n
        pc_horiz(x, C97::A, C97::B, AB, K1);
        R& y = w2[PH % 3];  // pair 1, row n-1
        pc_vert(y, w1[(PH + 1) % 3], w1[(PH + 2) % 3], x, C97::A, C97::B, AB, K1);
        pc_horiz(y, C97::G, C97::D, GD, K2);
        pc_vert(o, w2[(PH + 1) % 3], w2[(PH + 2) % 3], y, C97::G, C97::D, GD, K2);  // row n-2
        scale97(o);
        return o;
    }
};

// --- convolution --------------------------------------------------------------
// The whole CDF 9/7 analysis as one 1-D filter bank per axis: the polyphase
// matrix diag(zeta, 1/zeta) [V2 U2; P2 1] [V1 U1; P1 1] multiplied out at
// compile time from the lifting constants,
//   [s'; d'] = [A(z) B(z); C(z) D(z)] [s; d],
// A: taps -2..2 (symmetric), B: -2..1 (B_k = B_{-1-k}), C: -1..2 (C_k = C_{1-k}),
// D: -1..1 (symmetric), i.e. the 9-tap low-pass and 7-tap high-pass filters.
// A row streams through the horizontal bank (one exchange of pre-transform
// neighbours up to two quads away), and the vertical bank combines five rows
// of its result held in a ring of six registers rows.  As with the
// polyconvolution, the separable and non-separable convolution schemes of the
// paper coincide here.
struct LPoly9 {  // Laurent polynomial, coefficients of z^-4 .. z^4
    double c[9];
};
constexpr LPoly9 lp_term(int k, double v) {
    LPoly9 r{};
    r.c[k + 4] = v;
    return r;
}
constexpr LPoly9 lp_add(const LPoly9& x, const LPoly9& y) {
    LPoly9 r{};
    for (int i = 0; i < 9; ++i) r.c[i] = x.c[i] + y.c[i];
    return r;
}
constexpr LPoly9 lp_mul(const LPoly9& x, const LPoly9& y) {
    LPoly9 r{};
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            const int k = i + j - 4;
            if (k >= 0 && k < 9) r.c[k] += x.c[i] * y.c[j];
        }
    return r;
}
constexpr LPoly9 lp_scale(const LPoly9& x, double s) {
    LPoly9 r{};
    for (int i = 0; i < 9; ++i) r.c[i] = x.c[i] * s;
    return r;
}
struct Conv97 {
    static constexpr LPoly9 P1 = lp_add(lp_term(0, C97::Ad), lp_term(1, C97::Ad));   // a(1 + z)
    static constexpr LPoly9 U1 = lp_add(lp_term(0, C97::Bd), lp_term(-1, C97::Bd));  // b(1 + z^-1)
    static constexpr LPoly9 P2 = lp_add(lp_term(0, C97::Gd), lp_term(1, C97::Gd));
    static constexpr LPoly9 U2 = lp_add(lp_term(0, C97::Dd), lp_term(-1, C97::Dd));
    static constexpr LPoly9 V1 = lp_add(lp_term(0, 1.0), lp_mul(U1, P1));
    static constexpr LPoly9 V2 = lp_add(lp_term(0, 1.0), lp_mul(U2, P2));
    static constexpr LPoly9 A = lp_scale(lp_add(lp_mul(V2, V1), lp_mul(U2, P1)), C97::Zd);
    static constexpr LPoly9 B = lp_scale(lp_add(lp_mul(V2, U1), U2), C97::Zd);
    static constexpr LPoly9 C = lp_scale(lp_add(lp_mul(P2, V1), P1), 1.0 / C97::Zd);
    static constexpr LPoly9 D = lp_scale(lp_add(lp_mul(P2, U1), lp_term(0, 1.0)), 1.0 / C97::Zd);
    // distinct taps (index k + 4 is the coefficient of z^k)
    static constexpr float A0 = float(A.c[4]), A1 = float(A.c[5]), A2 = float(A.c[6]);
    static constexpr float B0 = float(B.c[4]), B1 = float(B.c[5]);  // B_0 = B_-1, B_1 = B_-2
    static constexpr float C0 = float(C.c[4]), C2 = float(C.c[6]);  // C_0 = C_1, C_2 = C_-1
    static constexpr float D0 = float(D.c[4]), D1 = float(D.c[5]);  // D_1 = D_-1
};

// values of the quads two to the left / right (QL >= 2)
template <class CT, int QL>
__device__ __forceinline__ void left2_of(const CT (&x)[QL], CT (&l)[QL]) {
    static_assert(QL >= 2, "two-quad neighbours come from the adjacent lane");
    const CT p0 = __shfl_up_sync(FULL, x[QL - 2], 1), p1 = __shfl_up_sync(FULL, x[QL - 1], 1);
    l[0] = p0;
    l[1] = p1;
#pragma unroll
    for (int q = 2; q < QL; ++q) l[q] = x[q - 2];
}
template <class CT, int QL>
__device__ __forceinline__ void right2_of(const CT (&x)[QL], CT (&r)[QL]) {
    static_assert(QL >= 2, "two-quad neighbours come from the adjacent lane");
    const CT n0 = __shfl_down_sync(FULL, x[0], 1), n1 = __shfl_down_sync(FULL, x[1], 1);
#pragma unroll
    for (int q = 0; q + 2 < QL; ++q) r[q] = x[q + 2];
    r[QL - 2] = n0;
    r[QL - 1] = n1;
}

// the horizontal bank on the pixel row (s, d) of every quad, in place
template <int QL>
__device__ __forceinline__ void cv_bank(float (&s)[QL], float (&d)[QL]) {
    using K = Conv97;
    float sl[QL], sr[QL], sll[QL], srr[QL], dl[QL], dr[QL], dll[QL];
    left_of(s, sl);
    right_of(s, sr);
    left2_of(s, sll);
    right2_of(s, srr);
    left_of(d, dl);
    right_of(d, dr);
    left2_of(d, dll);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const float lo = fmaf(K::A2, sll[q] + srr[q], fmaf(K::A1, sl[q] + sr[q], K::A0 * s[q])) +
                         fmaf(K::B1, dll[q] + dr[q], K::B0 * (dl[q] + d[q]));
        const float hi = fmaf(K::C2, sl[q] + srr[q], K::C0 * (s[q] + sr[q])) +
                         fmaf(K::D1, dl[q] + dr[q], K::D0 * d[q]);
        s[q] = lo;
        d[q] = hi;
    }
}

template <int QL>
struct Fwd97CV {
    static constexpr int LAG = 2;
    using CT = float;
    using R = Row<float, QL>;
    R hw[6], o;  // horizontal results of the last rows, ring indexed by phase
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 6; ++i) zero_row(hw[i]);
    }
    template <int PH>
    __device__ __forceinline__ R& slot() {
        return hw[PH % 6];
    }
    template <int PH>
    __device__ __forceinline__ R& step(int /*row*/) {
        using K = Conv97;
        R& x = hw[PH % 6];  // arrival n; output row r = n - 2
        cv_bank(x.c1, x.c2);
        cv_bank(x.c3, x.c4);
        const R& m2 = hw[(PH + 2) % 6];  // row r-2
        const R& m1 = hw[(PH + 3) % 6];  // row r-1
        const R& z0 = hw[(PH + 4) % 6];  // row r
        const R& p1 = hw[(PH + 5) % 6];  // row r+1
        const R& p2 = x;                 // row r+2
#pragma unroll
        for (int q = 0; q < QL; ++q) {
            // vertical bank on the columns (h1, h3) -> (c1, c3) and (h2, h4) -> (c2, c4)
            o.c1[q] = fmaf(K::A2, m2.c1[q] + p2.c1[q], fmaf(K::A1, m1.c1[q] + p1.c1[q], K::A0 * z0.c1[q])) +
                      fmaf(K::B1, m2.c3[q] + p1.c3[q], K::B0 * (m1.c3[q] + z0.c3[q]));
            o.c3[q] = fmaf(K::C2, m1.c1[q] + p2.c1[q], K::C0 * (z0.c1[q] + p1.c1[q])) +
                      fmaf(K::D1, m1.c3[q] + p1.c3[q], K::D0 * z0.c3[q]);
            o.c2[q] = fmaf(K::A2, m2.c2[q] + p2.c2[q], fmaf(K::A1, m1.c2[q] + p1.c2[q], K::A0 * z0.c2[q])) +
                      fmaf(K::B1, m2.c4[q] + p1.c4[q], K::B0 * (m1.c4[q] + z0.c4[q]));
            o.c4[q] = fmaf(K::C2, m1.c2[q] + p2.c2[q], K::C0 * (z0.c2[q] + p1.c2[q])) +
                      fmaf(K::D1, m1.c4[q] + p1.c4[q], K::D0 * z0.c4[q]);
        }
        return o;
    }
};

// --- non-separable convolution ------------------------------------------------
// The whole CDF 9/7 analysis as one step of 2-D filters, N = N^V N^H (Proposed
// Schemes): each output band is the sum of the 2-D convolutions of the four
// polyphase inputs with products of one vertical and one horizontal tap of
// the 1-D bank above (filters of 9x9, 9x7, 7x9 and 7x7 pixels), applied
// directly, with no intermediate result of either direction.  An arriving
// quad row is multiplied into the five output rows it reaches (a ring of six
// accumulator rows); its horizontal neighbours are fetched once and the
// pairs of equal horizontal taps added first.  144 FMA and 14 additions per
// quad, against about 70 operations of the separable bank.

// 1-D taps by offset k = input - output (quads): low-pass on the even (A) and
// odd (B) phase, high-pass on the even (C) and odd (D) phase
constexpr double nc_tap(int f, int k) {
    return f == 0 ? (k == 0 ? Conv97::A.c[4] : (k == 1 || k == -1) ? Conv97::A.c[5]
                                                   : (k == 2 || k == -2) ? Conv97::A.c[6] : 0.0)
         : f == 1 ? ((k == 0 || k == -1) ? Conv97::B.c[4] : (k == 1 || k == -2) ? Conv97::B.c[5] : 0.0)
         : f == 2 ? ((k == 0 || k == 1) ? Conv97::C.c[4] : (k == 2 || k == -1) ? Conv97::C.c[6] : 0.0)
                  : (k == 0 ? Conv97::D.c[4] : (k == 1 || k == -1) ? Conv97::D.c[5] : 0.0);
}
template <int F, int K>
struct NcV {
    static constexpr double v = nc_tap(F, K);
};

// one pixel row's horizontal terms, symmetric pairs added: a0..a2 for the
// low-pass taps on the even columns, b0, b1 on the odd ones; c0, c2 and d0,
// d1 likewise for the high-pass
template <int QL>
struct NcH {
    float a0[QL], a1[QL], a2[QL], b0[QL], b1[QL], c0[QL], c2[QL], d0[QL], d1[QL];
};
template <int QL>
__device__ __forceinline__ void nc_terms(const float (&s)[QL], const float (&d)[QL], NcH<QL>& t) {
    float sl[QL], sr[QL], sll[QL], srr[QL], dl[QL], dr[QL], dll[QL];
    left_of(s, sl);
    right_of(s, sr);
    left2_of(s, sll);
    right2_of(s, srr);
    left_of(d, dl);
    right_of(d, dr);
    left2_of(d, dll);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        t.a0[q] = s[q];
        t.a1[q] = sl[q] + sr[q];
        t.a2[q] = sll[q] + srr[q];
        t.b0[q] = dl[q] + d[q];
        t.b1[q] = dll[q] + dr[q];
        t.c0[q] = s[q] + sr[q];
        t.c2[q] = sl[q] + srr[q];
        t.d0[q] = d[q];
        t.d1[q] = dl[q] + dr[q];
    }
}
// acc += V * (horizontal low-pass of t), every product a compile-time constant
template <class V, int QL>
__device__ __forceinline__ void nc_low(float (&acc)[QL], const NcH<QL>& t) {
    if constexpr (V::v != 0.0) {
        constexpr float k0 = float(V::v * Conv97::A.c[4]), k1 = float(V::v * Conv97::A.c[5]),
                        k2 = float(V::v * Conv97::A.c[6]), k3 = float(V::v * Conv97::B.c[4]),
                        k4 = float(V::v * Conv97::B.c[5]);
#pragma unroll
        for (int q = 0; q < QL; ++q)
            acc[q] = fmaf(k4, t.b1[q], fmaf(k3, t.b0[q], fmaf(k2, t.a2[q], fmaf(k1, t.a1[q], fmaf(k0, t.a0[q], acc[q])))));
    }
}
template <class V, int QL>
__device__ __forceinline__ void nc_high(float (&acc)[QL], const NcH<QL>& t) {
    if constexpr (V::v != 0.0) {
        constexpr float k0 = float(V::v * Conv97::C.c[4]), k2 = float(V::v * Conv97::C.c[6]),
                        k3 = float(V::v * Conv97::D.c[4]), k4 = float(V::v * Conv97::D.c[5]);
#pragma unroll
        for (int q = 0; q < QL; ++q)
            acc[q] = fmaf(k4, t.d1[q], fmaf(k3, t.d0[q], fmaf(k2, t.c2[q], fmaf(k0, t.c0[q], acc[q]))));
    }
}
// the contribution of an arriving row (even pixel row e, odd pixel row o) to
// the output row K quad rows above it
template <int K, int QL>
__device__ __forceinline__ void nc_add(Row<float, QL>& r, const NcH<QL>& e, const NcH<QL>& o) {
    nc_low<NcV<0, K>>(r.c1, e);  // LL: vertical low-pass, even / odd row
    nc_low<NcV<1, K>>(r.c1, o);
    nc_high<NcV<0, K>>(r.c2, e);  // HL
    nc_high<NcV<1, K>>(r.c2, o);
    nc_low<NcV<2, K>>(r.c3, e);  // LH: vertical high-pass
    nc_low<NcV<3, K>>(r.c3, o);
    nc_high<NcV<2, K>>(r.c4, e);  // HH
    nc_high<NcV<3, K>>(r.c4, o);
}

template <int QL>
struct Fwd97NC {
    static constexpr int LAG = 2;
    using CT = float;
    using R = Row<float, QL>;
    R x, acc[6];  // the arriving row; output rows n-2 .. n+3 by phase
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 6; ++i) zero_row(acc[i]);
    }
    template <int PH>
    __device__ __forceinline__ R& slot() {
        return x;
    }
    template <int PH>
    __device__ __forceinline__ R& step(int /*row*/) {
        // arrival n reaches output rows n+2 (first) .. n-2 (last, complete now)
        zero_row(acc[(PH + 2) % 6]);
        NcH<QL> e, o;
        nc_terms(x.c1, x.c2, e);
        nc_terms(x.c3, x.c4, o);
        nc_add<-2>(acc[(PH + 2) % 6], e, o);
        nc_add<-1>(acc[(PH + 1) % 6], e, o);
        nc_add<0>(acc[PH % 6], e, o);
        nc_add<1>(acc[(PH + 5) % 6], e, o);
        nc_add<2>(acc[(PH + 4) % 6], e, o);
        return acc[(PH + 4) % 6];
    }
};

// the CDF 9/7 forward pipeline of a scheme
template <int SCHEME, int QL>
struct Fwd97Sel {
    using type = Fwd97<SCHEME, QL>;
};
template <int QL>
struct Fwd97Sel<SCHEME_POLYCONV, QL> {
    using type = Fwd97PC<QL>;
};
template <int QL>
struct Fwd97Sel<SCHEME_CONV, QL> {
    using type = Fwd97CV<QL>;
};
template <int QL>
struct Fwd97Sel<SCHEME_NSCONV, QL> {
    using type = Fwd97NC<QL>;
};
template <int SCHEME, int QL>
using Fwd97S = typename Fwd97Sel<SCHEME, QL>::type;

// inverse: unscale, then for each pair in reverse order S_{-U}, T_{-P}
template <int SCHEME, int QL>
struct Inv97 {
    static constexpr int LAG = 2;
    using CT = float;
    using R = Row<float, QL>;
    R rw[3];
    Carry3<QL> ka[2], kb[2];
    Carry2<float, QL> sa[2], sb[2];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 3; ++i) zero_row(rw[i]);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            zero_carry(ka[i]);
            zero_carry(kb[i]);
            zero_carry(sa[i]);
            zero_carry(sb[i]);
        }
    }
    template <int PH>
    __device__ __forceinline__ R& slot() {
        return rw[PH % 3];
    }
    template <int PH>
    __device__ __forceinline__ R& step(int /*row*/) {
        R& r0 = rw[PH % 3];
        R& r1 = rw[(PH + 2) % 3];
        R& r2 = rw[(PH + 1) % 3];
        constexpr int c = PH & 1, n = c ^ 1;
        unscale97(r0);
        if constexpr (SCHEME == SCHEME_NONSEP) {
            ns_update(r0, kb[c], kb[n], -C97::D, C97::DD);
            ns_predict(r1, r0, -C97::G, C97::GG);
            ns_update(r1, ka[c], ka[n], -C97::B, C97::BB);
            ns_predict(r2, r1, -C97::A, C97::AA);
        } else if constexpr (SCHEME == SCHEME_REDUCED) {
            rdi_update(r0, kb[c], kb[n], C97::D, C97::DD);
            rdi_predict_local(r0, C97::G);
            rdi_predict_exch(r1, r0, C97::G, C97::GG);
            rdi_update(r1, ka[c], ka[n], C97::B, C97::BB);
            rdi_predict_local(r1, C97::A);
            rdi_predict_exch(r2, r1, C97::A, C97::AA);
        } else {
            sp_sv(r0, sb[c], sb[n], -C97::D);
            sp_sh(r0, -C97::D);
            sp_tv(r1, r0, -C97::G);
            sp_th(r1, -C97::G);
            sp_sv(r1, sa[c], sa[n], -C97::B);
            sp_sh(r1, -C97::B);
            sp_tv(r2, r1, -C97::A);
            sp_th(r2, -C97::A);
        }
        return r2;
    }
};

// ==================================================== adjoint of CDF 9/7
// The forward operator with the whole-sample symmetric boundary is
// W = R F E: extend the level's input symmetrically (E), lift on the
// unbounded extended domain with no boundary cases (F), keep the
// coefficients inside (R).  Its transpose is W^T = E^T F^T R^T: the
// coefficient gradient placed on the extended domain with zeros outside (R^T),
// the transposed lifting with no boundary cases (F^T), and the fold E^T that
// adds the value of every extended position onto its whole-sample mirror.
// F^T is the transposed steps in reverse order: scaling (symmetric), then
// for each pair S_U^T and T_P^T.  Unweighted, U^T = b(1 + z) and
// P^T = a(1 + z^-1), so S_U^T is a spatial predict with coefficient b and
// T_P^T a spatial update with coefficient a, and the reduced split applies.
// Every output within four pixels of the image (two quads) can be nonzero;
// the kernels write those outside the image to a side buffer and fold them
// (adj_fold_kernel).
template <int QL>
struct Adj97 {
    static constexpr int LAG = 2;
    using CT = float;
    using R = Row<float, QL>;
    R rw[3];
    Carry3<QL> ka[2], kb[2];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 3; ++i) zero_row(rw[i]);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            zero_carry(ka[i]);
            zero_carry(kb[i]);
        }
    }
    template <int PH>
    __device__ __forceinline__ R& slot() {
        return rw[PH % 3];
    }
    template <int PH>
    __device__ __forceinline__ R& step(int /*row*/) {
        R& r0 = rw[PH % 3];
        R& r1 = rw[(PH + 2) % 3];
        R& r2 = rw[(PH + 1) % 3];
        constexpr int c = PH & 1, n = c ^ 1;
        scale97(r0);
        rd_predict(r1, r0, C97::D, C97::DD);
        rd_update(r1, ka[c], ka[n], C97::G, C97::GG);
        rd_predict(r2, r1, C97::B, C97::BB);
        rd_update(r2, kb[c], kb[n], C97::A, C97::AA);
        return r2;
    }
};

// ====================================================== integer CDF 5/3
// Reversible 5/3: d -= floor((s_l + s_r)/2), s += floor((d_l + d_r + 2)/4),
// in the separable order T^H, T^V, S^H, S^V (arithmetic shifts are floor).

// fused T_P = T_P^V T_P^H in one step: the neighbour below has its c2 taken
// after T^H, recomputed here from its pre-step values (the analogue of PP*).
template <int QL>
__device__ __forceinline__ void int_ns_predict(Row<int, QL>& X, const Row<int, QL>& D) {
    int r1[QL], r3[QL], dr1[QL];
    right_of(X.c1, r1);
    right_of(X.c3, r3);
    right_of(D.c1, dr1);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int c2n = X.c2[q] - ((X.c1[q] + r1[q]) >> 1);
        const int d2n = D.c2[q] - ((D.c1[q] + dr1[q]) >> 1);
        const int c4a = X.c4[q] - ((X.c3[q] + r3[q]) >> 1);
        X.c3[q] = X.c3[q] - ((X.c1[q] + D.c1[q]) >> 1);
        X.c4[q] = c4a - ((c2n + d2n) >> 1);
        X.c2[q] = c2n;
    }
}

// fused S_U = S_U^V S_U^H; the carry holds the row above after its update.
template <int QL>
__device__ __forceinline__ void int_ns_update(Row<int, QL>& X, const Carry2<int, QL>& C, Carry2<int, QL>& N) {
    int l2[QL], l4[QL];
    left_of(X.c2, l2);
    left_of(X.c4, l4);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        int c1 = X.c1[q] + ((l2[q] + X.c2[q] + 2) >> 2);
        const int c3 = X.c3[q] + ((l4[q] + X.c4[q] + 2) >> 2);
        c1 += (C.c3[q] + c3 + 2) >> 2;
        const int c2 = X.c2[q] + ((C.c4[q] + X.c4[q] + 2) >> 2);
        X.c1[q] = c1;
        X.c2[q] = c2;
        X.c3[q] = c3;
        N.c3[q] = c3;
        N.c4[q] = X.c4[q];
    }
}

template <int QL>
__device__ __forceinline__ void int_ns_update_inv(Row<int, QL>& X, const Carry2<int, QL>& C, Carry2<int, QL>& N) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        N.c3[q] = X.c3[q];
        N.c4[q] = X.c4[q];
        X.c2[q] -= (C.c4[q] + X.c4[q] + 2) >> 2;
        X.c1[q] -= (C.c3[q] + X.c3[q] + 2) >> 2;
    }
    int l2[QL], l4[QL];
    left_of(X.c2, l2);
    left_of(X.c4, l4);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c1[q] -= (l2[q] + X.c2[q] + 2) >> 2;
        X.c3[q] -= (l4[q] + X.c4[q] + 2) >> 2;
    }
}

template <int QL>
__device__ __forceinline__ void int_ns_predict_inv(Row<int, QL>& X, const Row<int, QL>& D) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c4[q] += (X.c2[q] + D.c2[q]) >> 1;
        X.c3[q] += (X.c1[q] + D.c1[q]) >> 1;
    }
    int r1[QL], r3[QL];
    right_of(X.c1, r1);
    right_of(X.c3, r3);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c4[q] += (X.c3[q] + r3[q]) >> 1;
        X.c2[q] += (X.c1[q] + r1[q]) >> 1;
    }
}

template <int QL>
__device__ __forceinline__ void int_sp_th(Row<int, QL>& X, int sgn) {
    int r1[QL], r3[QL];
    right_of(X.c1, r1);
    right_of(X.c3, r3);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c2[q] -= sgn * ((X.c1[q] + r1[q]) >> 1);
        X.c4[q] -= sgn * ((X.c3[q] + r3[q]) >> 1);
    }
}
template <int QL>
__device__ __forceinline__ void int_sp_tv(Row<int, QL>& X, const Row<int, QL>& D, int sgn) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c3[q] -= sgn * ((X.c1[q] + D.c1[q]) >> 1);
        X.c4[q] -= sgn * ((X.c2[q] + D.c2[q]) >> 1);
    }
}
template <int QL>
__device__ __forceinline__ void int_sp_sh(Row<int, QL>& X, int sgn) {
    int l2[QL], l4[QL];
    left_of(X.c2, l2);
    left_of(X.c4, l4);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c1[q] += sgn * ((l2[q] + X.c2[q] + 2) >> 2);
        X.c3[q] += sgn * ((l4[q] + X.c4[q] + 2) >> 2);
    }
}
template <int QL>
__device__ __forceinline__ void int_sp_sv(Row<int, QL>& X, const Carry2<int, QL>& C, Carry2<int, QL>& N, int sgn) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        X.c1[q] += sgn * ((C.c3[q] + X.c3[q] + 2) >> 2);
        X.c2[q] += sgn * ((C.c4[q] + X.c4[q] + 2) >> 2);
        N.c3[q] = X.c3[q];
        N.c4[q] = X.c4[q];
    }
}

template <int SCHEME, int QL>
struct Fwd53 {
    static constexpr int LAG = 1;
    using CT = int;
    using R = Row<int, QL>;
    R rw[2];
    Carry2<int, QL> k[2];
    __device__ __forceinline__ void init() {
        zero_row(rw[0]);
        zero_row(rw[1]);
        zero_carry(k[0]);
        zero_carry(k[1]);
    }
    template <int PH>
    __device__ __forceinline__ R& slot() {
        return rw[PH % 2];
    }
    template <int PH>
    __device__ __forceinline__ R& step(int /*row*/) {
        R& r0 = rw[PH % 2];
        R& r1 = rw[(PH + 1) % 2];
        constexpr int c = PH & 1, n = c ^ 1;
        if constexpr (SCHEME == SCHEME_SEP) {
            int_sp_th(r0, 1);
            int_sp_tv(r1, r0, 1);
            int_sp_sh(r1, 1);
            int_sp_sv(r1, k[c], k[n], 1);
        } else {
            int_ns_predict(r1, r0);
            int_ns_update(r1, k[c], k[n]);
        }
        return r1;
    }
};

template <int SCHEME, int QL>
struct Inv53 {
    static constexpr int LAG = 1;
    using CT = int;
    using R = Row<int, QL>;
    R rw[2];
    Carry2<int, QL> k[2];
    __device__ __forceinline__ void init() {
        zero_row(rw[0]);
        zero_row(rw[1]);
        zero_carry(k[0]);
        zero_carry(k[1]);
    }
    template <int PH>
    __device__ __forceinline__ R& slot() {
        return rw[PH % 2];
    }
    template <int PH>
    __device__ __forceinline__ R& step(int /*row*/) {
        R& r0 = rw[PH % 2];
        R& r1 = rw[(PH + 1) % 2];
        constexpr int c = PH & 1, n = c ^ 1;
        if constexpr (SCHEME == SCHEME_SEP) {
            int_sp_sv(r0, k[c], k[n], -1);
            int_sp_sh(r0, -1);
            int_sp_tv(r1, r0, -1);
            int_sp_th(r1, -1);
        } else {
            int_ns_update_inv(r0, k[c], k[n]);
            int_ns_predict_inv(r1, r0);
        }
        return r1;
    }
};

// ============================================================ DD 13/7 float
// The interpolating Deslauriers-Dubuc 13/7 wavelet: one lifting pair with the
// 4-tap predict P (cubic interpolation at the odd samples: weights 9/16 on
// the two nearest even samples, -1/16 on the next two, sign folded in) and
// the 4-tap update U (9/32, -1/32), no scaling step.  In quad terms P reads
// quads -1 .. +2 (near 0, +1; far -1, +2) and U reads quads -2 .. +1 (near
// -1, 0; far -2, +1); P* and U* are the same along columns.  A finished
// quad depends on input quads up to three away, so these pipelines declare a
// halo of four quads (which keeps a strip's first pixel a multiple of four)
// and three warm-up rows; a row leaves LAG = 3 rows after it arrived.
struct CDD {
    static constexpr float PN = -9.0f / 16.0f, PF = 1.0f / 16.0f;  // predict near / far
    static constexpr float UN = 9.0f / 32.0f, UF = -1.0f / 32.0f;  // update near / far
};

// P x along the row: near (x[q] + x[q+1]), far (x[q-1] + x[q+2])
template <int QL>
__device__ __forceinline__ void dd_ph(const float (&x)[QL], float (&o)[QL], float pn, float pf) {
    float l[QL], r[QL], rr[QL];
    left_of(x, l);
    right_of(x, r);
    right2_of(x, rr);
#pragma unroll
    for (int q = 0; q < QL; ++q) o[q] = fmaf(pf, l[q] + rr[q], pn * (x[q] + r[q]));
}
// U x along the row: near (x[q-1] + x[q]), far (x[q-2] + x[q+1])
template <int QL>
__device__ __forceinline__ void dd_uh(const float (&x)[QL], float (&o)[QL], float un, float uf) {
    float l[QL], ll[QL], r[QL];
    left_of(x, l);
    left2_of(x, ll);
    right_of(x, r);
#pragma unroll
    for (int q = 0; q < QL; ++q) o[q] = fmaf(uf, ll[q] + r[q], un * (l[q] + x[q]));
}
// the same along the column, from the rows a0 .. a3 (top to bottom) of the
// window: P* for the row a1 (a0 far, a1 a2 near, a3 far), U* for the row a2
__device__ __forceinline__ float dd_v(float a0, float a1, float a2, float a3, float near, float far) {
    return fmaf(far, a0 + a3, near * (a1 + a2));
}

// Spatial predict T_P of row m from the pre-step rows m-1 .. m+2 (w0 .. w3):
// the new (c1, c2, c3, c4) of row m.
template <int QL>
__device__ __forceinline__ void dd_ns_predict(const Row<float, QL>& w0, const Row<float, QL>& w1,
                                              const Row<float, QL>& w2, const Row<float, QL>& w3, Row<float, QL>& o,
                                              float pn, float pf) {
    float v1[QL], v2[QL], h1[QL], h3[QL], hv1[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        v1[q] = dd_v(w0.c1[q], w1.c1[q], w2.c1[q], w3.c1[q], pn, pf);  // P* c1
        v2[q] = dd_v(w0.c2[q], w1.c2[q], w2.c2[q], w3.c2[q], pn, pf);  // P* c2
    }
    dd_ph(w1.c1, h1, pn, pf);  // P c1
    dd_ph(w1.c3, h3, pn, pf);  // P c3
    dd_ph(v1, hv1, pn, pf);    // P P* c1
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        o.c1[q] = w1.c1[q];
        o.c2[q] = w1.c2[q] + h1[q];
        o.c3[q] = w1.c3[q] + v1[q];
        o.c4[q] = w1.c4[q] + (hv1[q] + v2[q] + h3[q]);
    }
}
// Spatial update S_U of row k from the pre-step rows k-2 .. k+1 (w0 .. w3).
template <int QL>
__device__ __forceinline__ void dd_ns_update(const Row<float, QL>& w0, const Row<float, QL>& w1,
                                             const Row<float, QL>& w2, const Row<float, QL>& w3, Row<float, QL>& o,
                                             float un, float uf) {
    float v3[QL], v4[QL], h2[QL], h4[QL], hv4[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        v3[q] = dd_v(w0.c3[q], w1.c3[q], w2.c3[q], w3.c3[q], un, uf);  // U* c3
        v4[q] = dd_v(w0.c4[q], w1.c4[q], w2.c4[q], w3.c4[q], un, uf);  // U* c4
    }
    dd_uh(w2.c2, h2, un, uf);  // U c2
    dd_uh(w2.c4, h4, un, uf);  // U c4
    dd_uh(v4, hv4, un, uf);    // U U* c4
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        o.c1[q] = w2.c1[q] + (h2[q] + v3[q] + hv4[q]);
        o.c2[q] = w2.c2[q] + v4[q];
        o.c3[q] = w2.c3[q] + h4[q];
        o.c4[q] = w2.c4[q];
    }
}

// --- reduced operations for DD 13/7 (Optimization Approach, Table 1) --------
// P = P0 + P1 with P0 = PN (the own quad's near tap) and the three other
// taps P1 = PN z + PF (z^-1 + z^2); U = U0 + U1 with U0 = UN and
// U1 = UN z^-1 + UF (z + z^-2).  The non-separable step keeps P1 (U1): 3 taps
// for each of P1 c1, P1* c1, P1* c2, P1 c3 and 9 for P1 P1* c1, i.e. 21
// operations; the constant parts follow as separable lifting inside the quad
// (T_{P0}^H, T_{P0}^V: 4 operations), which is Table 1's 2 x 21 + 8 = 50.
// P1 x along the row: PN x[q+1] + PF (x[q-1] + x[q+2])
template <int QL>
__device__ __forceinline__ void dd_p1h(const float (&x)[QL], float (&o)[QL], float pn, float pf) {
    float l[QL], r[QL], rr[QL];
    left_of(x, l);
    right_of(x, r);
    right2_of(x, rr);
#pragma unroll
    for (int q = 0; q < QL; ++q) o[q] = fmaf(pf, l[q] + rr[q], pn * r[q]);
}
// U1 x along the row: UN x[q-1] + UF (x[q-2] + x[q+1])
template <int QL>
__device__ __forceinline__ void dd_u1h(const float (&x)[QL], float (&o)[QL], float un, float uf) {
    float l[QL], ll[QL], r[QL];
    left_of(x, l);
    left2_of(x, ll);
    right_of(x, r);
#pragma unroll
    for (int q = 0; q < QL; ++q) o[q] = fmaf(uf, ll[q] + r[q], un * l[q]);
}

// T_{P1} then T_{P0}^H, T_{P0}^V of row m from the pre-step rows m-1 .. m+2.
template <int QL>
__device__ __forceinline__ void dd_rd_predict(const Row<float, QL>& w0, const Row<float, QL>& w1,
                                              const Row<float, QL>& w2, const Row<float, QL>& w3, Row<float, QL>& o,
                                              float pn, float pf) {
    float v1[QL], v2[QL], h1[QL], h3[QL], hv1[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        v1[q] = fmaf(pf, w0.c1[q] + w3.c1[q], pn * w2.c1[q]);  // P1* c1
        v2[q] = fmaf(pf, w0.c2[q] + w3.c2[q], pn * w2.c2[q]);  // P1* c2
    }
    dd_p1h(w1.c1, h1, pn, pf);  // P1 c1
    dd_p1h(w1.c3, h3, pn, pf);  // P1 c3
    dd_p1h(v1, hv1, pn, pf);    // P1 P1* c1
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const float c1 = w1.c1[q];
        const float c2 = fmaf(pn, c1, w1.c2[q] + h1[q]);           // T_{P1}, then T_{P0}^H on c2
        const float c3 = w1.c3[q] + v1[q];                         // T_{P1}
        const float c4 = fmaf(pn, c3, w1.c4[q] + (hv1[q] + v2[q] + h3[q]));  // T_{P1}, T_{P0}^H on c4
        o.c1[q] = c1;
        o.c2[q] = c2;
        o.c3[q] = fmaf(pn, c1, c3);                                 // T_{P0}^V
        o.c4[q] = fmaf(pn, c2, c4);
    }
}
// S_{U1} then S_{U0}^H, S_{U0}^V of row k from the pre-step rows k-2 .. k+1.
template <int QL>
__device__ __forceinline__ void dd_rd_update(const Row<float, QL>& w0, const Row<float, QL>& w1,
                                             const Row<float, QL>& w2, const Row<float, QL>& w3, Row<float, QL>& o,
                                             float un, float uf) {
    float v3[QL], v4[QL], h2[QL], h4[QL], hv4[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        v3[q] = fmaf(uf, w0.c3[q] + w3.c3[q], un * w1.c3[q]);  // U1* c3
        v4[q] = fmaf(uf, w0.c4[q] + w3.c4[q], un * w1.c4[q]);  // U1* c4
    }
    dd_u1h(w2.c2, h2, un, uf);  // U1 c2
    dd_u1h(w2.c4, h4, un, uf);  // U1 c4
    dd_u1h(v4, hv4, un, uf);    // U1 U1* c4
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const float c4 = w2.c4[q];
        const float c2 = w2.c2[q] + v4[q];                                    // S_{U1}
        const float c3 = fmaf(un, c4, w2.c3[q] + h4[q]);                      // S_{U1}, then S_{U0}^H on c3
        const float c1 = fmaf(un, c2, w2.c1[q] + (h2[q] + v3[q] + hv4[q]));   // S_{U1}, S_{U0}^H on c1
        o.c1[q] = fmaf(un, c3, c1);                                           // S_{U0}^V
        o.c2[q] = fmaf(un, c4, c2);
        o.c3[q] = c3;
        o.c4[q] = c4;
    }
}

// Separable steps.  Row-local: T_P^H (c2 += P c1, c4 += P c3) and S_U^H
// (c1 += U c2, c3 += U c4), in place.
template <int QL>
__device__ __forceinline__ void dd_sp_th(Row<float, QL>& x, float pn, float pf) {
    float h1[QL], h3[QL];
    dd_ph(x.c1, h1, pn, pf);
    dd_ph(x.c3, h3, pn, pf);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        x.c2[q] += h1[q];
        x.c4[q] += h3[q];
    }
}
template <int QL>
__device__ __forceinline__ void dd_sp_sh(Row<float, QL>& x, float un, float uf) {
    float h2[QL], h4[QL];
    dd_uh(x.c2, h2, un, uf);
    dd_uh(x.c4, h4, un, uf);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        x.c1[q] += h2[q];
        x.c3[q] += h4[q];
    }
}
// Column steps into o: T_P^V of row m from rows m-1 .. m+2 (c3 += P* c1,
// c4 += P* c2) and S_U^V of row k from rows k-2 .. k+1 (c1 += U* c3,
// c2 += U* c4).
template <int QL>
__device__ __forceinline__ void dd_sp_tv(const Row<float, QL>& w0, const Row<float, QL>& w1, const Row<float, QL>& w2,
                                         const Row<float, QL>& w3, Row<float, QL>& o, float pn, float pf) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        o.c1[q] = w1.c1[q];
        o.c2[q] = w1.c2[q];
        o.c3[q] = w1.c3[q] + dd_v(w0.c1[q], w1.c1[q], w2.c1[q], w3.c1[q], pn, pf);
        o.c4[q] = w1.c4[q] + dd_v(w0.c2[q], w1.c2[q], w2.c2[q], w3.c2[q], pn, pf);
    }
}
template <int QL>
__device__ __forceinline__ void dd_sp_sv(const Row<float, QL>& w0, const Row<float, QL>& w1, const Row<float, QL>& w2,
                                         const Row<float, QL>& w3, Row<float, QL>& o, float un, float uf) {
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        o.c1[q] = w2.c1[q] + dd_v(w0.c3[q], w1.c3[q], w2.c3[q], w3.c3[q], un, uf);
        o.c2[q] = w2.c2[q] + dd_v(w0.c4[q], w1.c4[q], w2.c4[q], w3.c4[q], un, uf);
        o.c3[q] = w2.c3[q];
        o.c4[q] = w2.c4[q];
    }
}

// Forward.  Arrival n (phase PH) lands in a[PH]; the first step runs on row
// n-2 from the arrived rows n-3 .. n into b[(PH+4) % 6], the second on row
// n-3 from b's rows n-5 .. n-2 into the output.  Rings of six rows, indexed by
// the phase, so that no row is copied.
template <int SCHEME, int QL>
struct Fwd137 {
    static constexpr int LAG = 3, HALO = 4, WARM = 3;
    using CT = float;
    using R = Row<float, QL>;
    R a[6], b[6], o;
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            zero_row(a[i]);
            zero_row(b[i]);
        }
    }
    template <int PH>
    __device__ __forceinline__ R& slot() {
        return a[PH];
    }
    template <int PH>
    __device__ __forceinline__ R& step(int /*row*/) {
        constexpr int M3 = (PH + 3) % 6, M2 = (PH + 4) % 6, M1 = (PH + 5) % 6, M5 = (PH + 1) % 6;
        if constexpr (SCHEME == SCHEME_SEP) {
            dd_sp_th(a[PH], CDD::PN, CDD::PF);  // rows enter after their T_P^H
            dd_sp_tv(a[M3], a[M2], a[M1], a[PH], b[M2], CDD::PN, CDD::PF);
            dd_sp_sh(b[M2], CDD::UN, CDD::UF);
            dd_sp_sv(b[M5], b[(PH + 2) % 6], b[M3], b[M2], o, CDD::UN, CDD::UF);
        } else if constexpr (SCHEME == SCHEME_REDUCED) {
            dd_rd_predict(a[M3], a[M2], a[M1], a[PH], b[M2], CDD::PN, CDD::PF);
            dd_rd_update(b[M5], b[(PH + 2) % 6], b[M3], b[M2], o, CDD::UN, CDD::UF);
        } else {
            dd_ns_predict(a[M3], a[M2], a[M1], a[PH], b[M2], CDD::PN, CDD::PF);
            dd_ns_update(b[M5], b[(PH + 2) % 6], b[M3], b[M2], o, CDD::UN, CDD::UF);
        }
        return o;
    }
};

// Inverse: arrival n (coefficients) lands in a[PH]; S_U undone on row n-1
// from the rows n-3 .. n into b[(PH+5) % 6], then T_P undone on row n-3 from
// b's rows n-4 .. n-1 into the output.
template <int SCHEME, int QL>
struct Inv137 {
    static constexpr int LAG = 3, HALO = 4, WARM = 3;
    using CT = float;
    using R = Row<float, QL>;
    R a[6], b[6], o;
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            zero_row(a[i]);
            zero_row(b[i]);
        }
    }
    template <int PH>
    __device__ __forceinline__ R& slot() {
        return a[PH];
    }
    template <int PH>
    __device__ __forceinline__ R& step(int /*row*/) {
        constexpr int M1 = (PH + 5) % 6, M2 = (PH + 4) % 6, M3 = (PH + 3) % 6, M4 = (PH + 2) % 6;
        if constexpr (SCHEME == SCHEME_SEP) {
            // S_U^V then S_U^H undone on row n-1, T_P^V then T_P^H on row n-3
            dd_sp_sv(a[M3], a[M2], a[M1], a[PH], b[M1], -CDD::UN, -CDD::UF);
            dd_sp_sh(b[M1], -CDD::UN, -CDD::UF);
            dd_sp_tv(b[M4], b[M3], b[M2], b[M1], o, -CDD::PN, -CDD::PF);
            dd_sp_th(o, -CDD::PN, -CDD::PF);
        } else {
            dd_ns_update(a[M3], a[M2], a[M1], a[PH], b[M1], -CDD::UN, -CDD::UF);
            dd_ns_predict(b[M4], b[M3], b[M2], b[M1], o, -CDD::PN, -CDD::PF);
        }
        return o;
    }
};

}  // namespace dwt2
