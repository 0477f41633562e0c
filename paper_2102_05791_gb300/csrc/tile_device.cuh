// Device functions of the tiled HVP shared by the per-iteration tile kernel
// (elem_kernels.cu) and the cooperative CG kernel (cg_coop.cu): one element's
// dP(dF) from its record, the corner-force stores, and one local vertex's
// fixed-order corner sum with its per-vertex terms.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "elem_math.cuh"
#include "internal.h"

namespace softsim {

// Corner forces of one element into its record (slots corner*D + i; corner
// 0 takes minus the column sum of G), written as pairs: 8-byte (FP32) or
// 16-byte (FP64) stores.  rec must be aligned to the pair size.
template <typename T, int D>
__device__ __forceinline__ void store_corners(T *rec, const T G[D][D])
{
    T out[(D + 1) * D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            out[(j + 1) * D + i] = G[i][j];
            s += G[i][j];
        }
        out[i] = -s;
    }
#pragma unroll
    for (int q = 0; q < (D + 1) * D / 2; ++q) {
        if constexpr (sizeof(T) == 4)
            reinterpret_cast<float2 *>(rec)[q] = make_float2(out[2 * q], out[2 * q + 1]);
        else
            reinterpret_cast<double2 *>(rec)[q] = make_double2(out[2 * q], out[2 * q + 1]);
    }
}

// Sum of the corners touching a local vertex in a fixed order: the entries
// of its incidence list at even and at odd positions are summed as two
// independent chains (two loads in flight per step), then added (inc points
// at the tile's incidence block, each entry the offset of a corner's D
// values among the tile's element records; w is the vertex's lv_inc word).
template <typename T, int D>
__device__ __forceinline__ void gather_corners(const uint16_t *inc, uint32_t w, const T *scr, T acc[D])
{
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = T(0);
    const int s0 = (int)(w & 0xffffu), n = (int)((w >> 16) & kLvCountMask);
    T acc1[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc1[c] = T(0);
    int s = s0;
    for (; s + 1 < s0 + n; s += 2) {
        const T *p = scr + inc[s], *q = scr + inc[s + 1];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            acc[c] += p[c];
            acc1[c] += q[c];
        }
    }
    if (s < s0 + n) {
        const T *p = scr + inc[s];
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] += p[c];
    }
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] += acc1[c];
}

// One element of the HVP: reads the element's record (pair loads) and the
// staged u and v of its vertices, evaluates G = W dP(dF) Dm^-T plus the
// muscle term, adds v_e . (H_e v_e) to qsum (CG), and writes the element's
// corner forces to out + corner_base(le) (out = rec overwrites the record in
// place; a separate buffer of the same stride keeps the record).
template <typename T, int D, bool CG, bool SPRING, int RS>
__device__ __forceinline__ void hvp_element(const T *rec, int le, uint32_t cword, const T *suv, const Phys &ph,
                                            T mu, T lam, T sel, T kk, T &qsum, T *out)
{
    constexpr int NF = hvp_fields(D, SPRING);
    int lid[D + 1];
    unpack<D>(cword, lid);
    // Dm^-1, g and W first (for the contractile muscle that includes the
    // activation); the spring's fiber and activation where they are used
    constexpr int N1 = (FI<D>::W + 2) / 2 * 2;
    T rv[RS];
    load_pairs<T, N1>(rec, rv);
    T B[D][D], Du[D][D], Dv[D][D], F[D][D], dF[D][D], C[D][D], dC[D][D], gv[D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) B[i][j] = rv[FI<D>::B + i * D + j];
#pragma unroll
    for (int i = 0; i < D; ++i) gv[i] = rv[FI<D>::G + i];
    const T W = rv[FI<D>::W] * sel;
    if constexpr (sizeof(T) == 4 && D == 3) {
        // paired FP32 arithmetic (__fadd2_rn / __ffma2_rn: two lanes per
        // instruction), the same operations in the same order as the scalar
        // form below, so this step's results are bitwise the same: a staged vertex is
        // the pairs (u0, u1), (u2, v0), (v1, v2), so the edges come as pairs
        // (Du0k, Du1k), (Du2k, Dv0k), (Dv1k, Dv2k), and F = I + Du B and
        // dF = Dv B as pairs (F0j, F1j), (F2j, dF0j), (dF1j, dF2j) with B[k][j]
        // on both lanes (27 paired FMAs instead of 54)
        const float2 *sp = reinterpret_cast<const float2 *>(suv);
        const float2 a0 = sp[3 * lid[0]], b0 = sp[3 * lid[0] + 1], c0 = sp[3 * lid[0] + 2];
        const float2 na0 = make_float2(-a0.x, -a0.y), nb0 = make_float2(-b0.x, -b0.y),
                     nc0 = make_float2(-c0.x, -c0.y);
        float2 P1[3], P2[3], P3[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int q = 3 * lid[k + 1];
            P1[k] = __fadd2_rn(sp[q], na0);
            P2[k] = __fadd2_rn(sp[q + 1], nb0);
            P3[k] = __fadd2_rn(sp[q + 2], nc0);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float2 x = make_float2(j == 0 ? 1.0f : 0.0f, j == 1 ? 1.0f : 0.0f);
            float2 y = make_float2(j == 2 ? 1.0f : 0.0f, 0.0f);
            float2 z = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float2 bb = make_float2(B[k][j], B[k][j]);
                x = __ffma2_rn(P1[k], bb, x);
                y = __ffma2_rn(P2[k], bb, y);
                z = __ffma2_rn(P3[k], bb, z);
            }
            F[0][j] = x.x;
            F[1][j] = x.y;
            F[2][j] = y.x;
            dF[0][j] = y.y;
            dF[1][j] = z.x;
            dF[2][j] = z.y;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Du[0][k] = P1[k].x;
            Du[1][k] = P1[k].y;
            Du[2][k] = P2[k].x;
            Dv[0][k] = P2[k].y;
            Dv[1][k] = P3[k].x;
            Dv[2][k] = P3[k].y;
        }
    } else {
        edges_uv<T, D>(suv, lid, Du, Dv);
        mul<T, D>(Du, B, F, true);
        mul<T, D>(Dv, B, dF, false);
    }
    cof<T, D>(F, C);
    dcof<T, D>(F, dF, dC);
    const T J = detF<T, D>(F, C);
    T dJ = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) dJ += C[i][j] * dF[i][j];
    T l, cc, cp;
    log_terms<T>(ph.log_mode, mu, lam, J, l, cc, cp);
    const T cpdJ = cp * dJ;
    T dvg[D];  // (d2psi_m/dq2) dq with dq = dF f = Dv g
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) s += Dv[i][k] * gv[k];
        dvg[i] = s;
    }
    if constexpr (N1 < RS) load_pairs<T, RS - N1>(rec + N1, rv + N1);
    const T aval = rv[NF];
    if constexpr (SPRING) {  // spring, with q = F f = f + Du g
        T q[D], s2 = T(0), qdq = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            T s = rv[FI<D>::F + i];
#pragma unroll
            for (int k = 0; k < D; ++k) s += Du[i][k] * gv[k];
            q[i] = s;
            s2 += s * s;
            qdq += s * dvg[i];
        }
        T c1, c2;
        spring_terms<T>(W != T(0), kk, aval, sqrt(s2), c1, c2);
#pragma unroll
        for (int i = 0; i < D; ++i) dvg[i] = c1 * dvg[i] + c2 * qdq * q[i];
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) dvg[i] *= kk * aval;
    }
    // G = W (dP Dm^-T + dvg g^T), with W folded into the coefficients of dP
    // and into dvg: dP = mu dF + c'(J) dJ cof F + c(J) dcof(F)[dF] formed once
    // per row entry, then multiplied by B^T
    const T muW = mu * W, cpW = cpdJ * W, ccW = cc * W;
    T M[D][D];
    T G[D][D];
    if constexpr (sizeof(T) == 4 && D == 3) {
        // rows 1 and 2 of M and G as pairs (dF rows 1 and 2 already are one),
        // row 0 scalar, in one fixed FMA order; p.Ap accumulated column by
        // column as G is formed, so each Dv entry dies once used
#pragma unroll
        for (int i = 0; i < D; ++i) dvg[i] *= W;
        const float2 muW2 = make_float2(muW, muW), cpW2 = make_float2(cpW, cpW), ccW2 = make_float2(ccW, ccW);
        float2 m12[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            M[0][k] = fmaf(ccW, dC[0][k], fmaf(cpW, C[0][k], muW * dF[0][k]));
            m12[k] = __ffma2_rn(ccW2, make_float2(dC[1][k], dC[2][k]),
                                __ffma2_rn(cpW2, make_float2(C[1][k], C[2][k]),
                                           __fmul2_rn(muW2, make_float2(dF[1][k], dF[2][k]))));
        }
        const float2 dv12 = make_float2(dvg[1], dvg[2]);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float s = dvg[0] * gv[j];
            float2 s12 = __fmul2_rn(dv12, make_float2(gv[j], gv[j]));
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                s = fmaf(M[0][k], B[j][k], s);
                s12 = __ffma2_rn(m12[k], make_float2(B[j][k], B[j][k]), s12);
            }
            G[0][j] = s;
            G[1][j] = s12.x;
            G[2][j] = s12.y;
            if (CG) {  // v_e . (H_e v_e) = Dv : G, column by column
                qsum += Dv[0][j] * G[0][j];
                qsum += Dv[1][j] * G[1][j];
                qsum += Dv[2][j] * G[2][j];
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            dvg[i] *= W;
#pragma unroll
            for (int k = 0; k < D; ++k) M[i][k] = muW * dF[i][k] + cpW * C[i][k] + ccW * dC[i][k];
        }
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                T s = dvg[i] * gv[j];
#pragma unroll
                for (int k = 0; k < D; ++k) s += M[i][k] * B[j][k];
                G[i][j] = s;
            }
    }
    if (CG && !(sizeof(T) == 4 && D == 3)) {
        // sum over corners of v_k . f_k = sum_j Dv[:,j] . G[:,j]
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) qsum += Dv[i][j] * G[i][j];
    }
    store_corners<T, D>(out + corner_base(le), G);  // the element's own corner block only
}

// One local vertex of the HVP: adds its corners in fixed order, adds the
// per-vertex terms (contact curvature, inertia, friction) where it owns
// them, and writes A v (single-tile vertex, masked) or its halo partial; the
// owner's vertex terms of p.Ap go to dot (CG).  uv: the vertex's staged
// record [u (D), v (D)].
template <typename T, int D, bool CG>
__device__ __forceinline__ void hvp_vertex(int code, uint32_t linc, int64_t gid, const T *uv, const uint16_t *sInc,
                                           const T *sRec, const VertDev &vd, const Phys &ph, T *__restrict__ y,
                                           T *__restrict__ hp, T &dot)
{
    if (code == LV_PAD) return;
    T acc[D];
    gather_corners<T, D>(sInc, linc, sRec, acc);
    const bool contact = ph.contact != 0, dyn = ph.dyn != 0;
    const bool interior = code == LV_INTERIOR;
    const bool owner = CG && (interior || (code & 1));  // counts the vertex terms of p.Ap
    if ((interior || owner) && (contact || dyn)) {
        T kcv = T(0), m = T(0), mh = T(0);  // contact curvature and inertia (+ friction) diagonals
        if (contact) {
            const double yy = vd.X[gid * D + 1] + (double)uv[1];
            const double pen = yy < 0.0 ? -yy : 0.0;
            const double d2 = pen > 0.0 ? ph.cpow * (ph.cpow - 1) * ph.kc * (ph.cpow == 2 ? 1.0 : pen) : 0.0;
            kcv = T(ph.s_el * d2);
        }
        if (dyn) {
            m = T(vd.mass[gid]);
            mh = ph.fw ? m + T(ph.fw[gid]) : m;  // friction stiffens the horizontal axes
        }
        T dv[D];
#pragma unroll
        for (int c = 0; c < D; ++c) dv[c] = (c == 1 ? m + kcv : mh) * uv[D + c];
        if (interior)
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] += dv[c];
        if (owner)
#pragma unroll
            for (int c = 0; c < D; ++c) dot += dv[c] * uv[D + c];
    }
    if (interior) {
        const bool fx = (linc & kLvPinned) != 0;
#pragma unroll
        for (int c = 0; c < D; ++c) y[gid * D + c] = fx ? T(0) : acc[c];
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) hp[(int64_t)(code >> 1) * D + c] = acc[c];
    }
}

}  // namespace softsim
