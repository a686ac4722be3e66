// The nonlocal (Kleinman-Bylander) part of the fused Chebyshev step on one unit of consecutive grid
// points held in shared memory (an xy plane, a group of x rows, or a CTA's rows of a cluster plane):
// the projections staged per slot, the apply colour by colour, and the per-slot partial projections
// of the step's output.  Unit point o (0 <= o < rows * N) is at sm[unit_pos(o)], by default
// sm[(o / N) * P + (o % N)].
// The tables are those of KBDev (slots, colours and entries per unit).
#pragma once
#include "fft_smem.cuh"
#include "grid_common.cuh"
#include "sgw_internal.cuh"

namespace sgw {

// Position in shared memory of unit point o = y N + x (row y, column x) at row pitch P.  LAYOUT 0:
// natural, y P + x.  LAYOUT 1 (N = 288, the two-stage row transforms): a row is 16 groups of 19
// slots, column x at 19 (x mod 16) + x div 16, the order in which the 16 x 18 transforms leave it.
template <int N, int P, int LAYOUT>
__device__ __forceinline__ int unit_pos_yx(int y, int x) {
    if constexpr (LAYOUT == 1) {
        static_assert(N == 288 && P >= 304, "layout 1 is the 288-point row in 16 groups of 19");
        return y * P + 19 * (x & 15) + (x >> 4);
    } else {
        return y * P + x;
    }
}
template <int N, int P, int LAYOUT>
__device__ __forceinline__ int unit_pos(int o) {
    return unit_pos_yx<N, P, LAYOUT>(o / N, o % N);
}

// E-weighted projector coefficients of the unit's slots into shared memory: kcs[4 s + p] for the
// unit's s-th slot and projector p.
template <int NT>
__device__ __forceinline__ void kb_stage_coeffs(const StepArgs& a, const float2* __restrict__ kc, int u, float2* kcs) {
    const int s0 = __ldg(a.plane_off + u), ns = __ldg(a.plane_off + u + 1) - s0;
    for (int i = threadIdx.x; i < 4 * ns; i += NT) kcs[i] = kc[__ldg(a.slot_atom + s0 + i / 4) * 4 + (i & 3)];
}

// sm += sum_ap beta_ap E_ap <beta_ap|b1> over the unit, colour by colour (slots of one colour touch
// disjoint points, so each point is updated by one thread at a time; no atomics, fixed order).
// Call after a barrier that made sm and kcs visible; returns after a barrier.
template <int N, int P, int NT, int LAYOUT = 0>
__device__ __forceinline__ void kb_apply_unit(const StepArgs& a, int u, const float2* kcs, float2* sm) {
    const int* col = a.kbe_col + (size_t)u * (a.max_colors + 1);
    for (int c = 0; c < a.max_colors; ++c) {
        const int e0 = __ldg(col + c), e1 = __ldg(col + c + 1);
        if (e0 == e1) break;                  // a unit's colours are used from 0 upwards
        for (int e = e0 + threadIdx.x; e < e1; e += NT) {
            const unsigned os = __ldg(a.kbe_os + e);
            const float4 be = __ldg(a.kbe_beta + e);
            const int o = (int)(os & 0xffffu), sl = (int)(os >> 16);
            const float4 c01 = *reinterpret_cast<const float4*>(kcs + 4 * sl);
            const float4 c23 = *reinterpret_cast<const float4*>(kcs + 4 * sl + 2);
            float2& hv = sm[unit_pos<N, P, LAYOUT>(o)];
            hv.x += be.x * c01.x + be.y * c01.z + be.z * c23.x + be.w * c23.z;
            hv.y += be.x * c01.y + be.y * c01.w + be.z * c23.y + be.w * c23.w;
        }
        __syncthreads();
    }
}

// Partial projections of the unit's values in sm (positions by unit_pos): kbp[b][slot][p] = sum over the slot's points of
// beta_ap(r) sm(r); one warp per slot, lanes strided over the points, fixed-order warp reduction.
template <int N, int P, int NT, int LAYOUT = 0>
__device__ __forceinline__ void kb_project_unit(const StepArgs& a, int u, int b, const float2* sm) {
    const int sb = __ldg(a.plane_off + u), s1 = __ldg(a.plane_off + u + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = sb + warp; k < s1; k += NT / 32) {
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int e1 = __ldg(a.kbe_slot_end + k);
        for (int e = __ldg(a.kbe_slot_beg + k) + lane; e < e1; e += 32) {
            const int o = (int)(__ldg(a.kbe_os + e) & 0xffffu);
            const float2 v = sm[unit_pos<N, P, LAYOUT>(o)];
            const float4 be = __ldg(a.kbe_beta + e);
            acc[0] += be.x * v.x; acc[1] += be.x * v.y;
            acc[2] += be.y * v.x; acc[3] += be.y * v.y;
            acc[4] += be.z * v.x; acc[5] += be.z * v.y;
            acc[6] += be.w * v.x; acc[7] += be.w * v.y;
        }
        const float r = warp_reduce_scatter8(acc, lane);
        if ((lane & 3) == 0) reinterpret_cast<float*>(a.kbp + ((size_t)b * a.total_slots + k) * 4)[lane >> 2] = r;
    }
}

// The pointwise part of the fused step on ROWS x N unit points starting at global offset `off`
// (vector b's unit; sm holds H_kin b1 + V_NL b1 at pitch P): out = cpsi psi + ch alpha (h + (V - Ebar) b1
// [+ dv b1_partner]) + c2 b2, written to global memory and back into sm.  STREAM: b1, psi, b2 read and
// out written with evict-first caching.
template <int N, int ROWS, int P, int NT, int UNROLL = 2, int LAYOUT = 0, bool STREAM = false>
__device__ __forceinline__ void step_pointwise(const StepArgs& a, const VecInfo& inf, size_t off, size_t uoff,
                                               float2* sm) {
    constexpr size_t NG = (size_t)N * N * N;
    const float* V = a.vpot + (size_t)inf.vrow * NG + uoff;
    const float* dV = (a.dvpot != nullptr && inf.dvrow >= 0) ? a.dvpot + (size_t)inf.dvrow * NG + uoff : nullptr;
    const float2* bp = (dV != nullptr) ? a.b1 + (size_t)inf.partner * NG + uoff : nullptr;
    const float2 cpsi = a.coef.cpsi[inf.cset], ch = a.coef.ch[inf.cset], c2 = a.coef.c2[inf.cset];
    const float ebar = a.ebar, alpha = a.alpha;
#pragma unroll UNROLL
    for (int q = threadIdx.x; q < ROWS * N / 2; q += NT) {
        const int y = q / (N / 2), x = 2 * (q % (N / 2));
        const int o = y * N + x;
        // x is even: x + 1 sits one slot further (layout 0) or one group of 19 further (layout 1)
        const int sp = unit_pos_yx<N, P, LAYOUT>(y, x), sp1 = sp + (LAYOUT == 1 ? 19 : 1);
        float2 h0 = sm[sp], h1 = sm[sp1];
        const float4 bb = STREAM ? ldcs4(a.b1 + off + o) : ld4(a.b1 + off + o);
        const float2 v = __ldg(reinterpret_cast<const float2*>(V + o));
        h0.x += (v.x - ebar) * bb.x;
        h0.y += (v.x - ebar) * bb.y;
        h1.x += (v.y - ebar) * bb.z;
        h1.y += (v.y - ebar) * bb.w;
        if (dV != nullptr) {
            const float2 d = __ldg(reinterpret_cast<const float2*>(dV + o));
            const float4 pb = ld4(bp + o);            // the partner's b1: another vector's launch reads it too
            h0.x += d.x * pb.x;
            h0.y += d.x * pb.y;
            h1.x += d.y * pb.z;
            h1.y += d.y * pb.w;
        }
        float2 o0 = cmul(ch, cscale(h0, alpha)), o1 = cmul(ch, cscale(h1, alpha));
        if (a.psi != nullptr) {
            const float4 pp = STREAM ? ldcs4(a.psi + off + o) : ld4(a.psi + off + o);
            o0 = cadd(o0, cmul(cpsi, make_float2(pp.x, pp.y)));
            o1 = cadd(o1, cmul(cpsi, make_float2(pp.z, pp.w)));
        }
        if (a.b2 != nullptr) {
            const float4 b2 = STREAM ? ldcs4(a.b2 + off + o) : ld4(a.b2 + off + o);
            o0 = cadd(o0, cmul(c2, make_float2(b2.x, b2.y)));
            o1 = cadd(o1, cmul(c2, make_float2(b2.z, b2.w)));
        }
        if (STREAM)
            stcs4(a.out + off + o, o0, o1);
        else
            st4(a.out + off + o, o0, o1);
        sm[sp] = o0;
        sm[sp1] = o1;
    }
}

}  // namespace sgw
