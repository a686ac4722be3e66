// Register DFTs of length 16, 9 and 18 and the 288-point twiddle lookup used by the two-stage
// 288 = 16 x 18 transforms of the 288 grid (line passes and the row step).
#pragma once
#include "fft_smem.cuh"

namespace sgw {

// exp(dir 2 pi i m / M) as (c, dir s)
template <int DIR>
__device__ __forceinline__ float2 rot(float2 v, float c, float s) {
    return cmul(v, make_float2(c, DIR * s));
}

// In-place 16-point DFT of v[0..15] with exp(dir 2 pi i n k / 16): 4 x 4, n = 4 a + b, k = c + 4 d.
template <int DIR>
__device__ __forceinline__ void dft16(float2* v) {
    constexpr float C1 = 0.923879532511286756f, S1 = 0.382683432365089772f;   // cos, sin (pi / 8)
    constexpr float R = 0.707106781186547524f;                                // 1 / sqrt 2
    float2 t[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
#pragma unroll
        for (int a = 0; a < 4; ++a) t[b][a] = v[4 * a + b];
        Dft<4, DIR>::run(t[b]);
    }
    // W16^(b c): exponents 1 2 3 / 2 4 6 / 3 6 9
    t[1][1] = rot<DIR>(t[1][1], C1, S1);
    t[1][2] = rot<DIR>(t[1][2], R, R);
    t[1][3] = rot<DIR>(t[1][3], S1, C1);
    t[2][1] = rot<DIR>(t[2][1], R, R);
    t[2][2] = mul_i<DIR>(t[2][2]);
    t[2][3] = rot<DIR>(t[2][3], -R, R);
    t[3][1] = rot<DIR>(t[3][1], S1, C1);
    t[3][2] = rot<DIR>(t[3][2], -R, R);
    t[3][3] = rot<DIR>(t[3][3], -C1, -S1);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float2 s[4] = {t[0][c], t[1][c], t[2][c], t[3][c]};
        Dft<4, DIR>::run(s);
#pragma unroll
        for (int d = 0; d < 4; ++d) v[c + 4 * d] = s[d];
    }
}

// In-place 9-point DFT of v[0..8]: 3 x 3, n = c + 3 e, k = a + 3 b.
template <int DIR>
__device__ __forceinline__ void dft9(float2* v) {
    constexpr float C1 = 0.766044443118978035f, S1 = 0.642787609686539326f;   // 2 pi / 9
    constexpr float C2 = 0.173648177666930349f, S2 = 0.984807753012208059f;   // 4 pi / 9
    constexpr float C4 = -0.939692620785908384f, S4 = 0.342020143325668733f;  // 8 pi / 9
    float2 t[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        t[c][0] = v[c];
        t[c][1] = v[c + 3];
        t[c][2] = v[c + 6];
        Dft<3, DIR>::run(t[c]);
    }
    // W9^(c a): exponents 1 2 / 2 4
    t[1][1] = rot<DIR>(t[1][1], C1, S1);
    t[1][2] = rot<DIR>(t[1][2], C2, S2);
    t[2][1] = rot<DIR>(t[2][1], C2, S2);
    t[2][2] = rot<DIR>(t[2][2], C4, S4);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float2 s[3] = {t[0][a], t[1][a], t[2][a]};
        Dft<3, DIR>::run(s);
        v[a] = s[0];
        v[a + 3] = s[1];
        v[a + 6] = s[2];
    }
}

// In-place 18-point DFT of v[0..17]: 2 x 9, n = 9 a + b, k = c + 2 d.
template <int DIR>
__device__ __forceinline__ void dft18(float2* v) {
    // cos, sin (2 pi b / 18), b = 1..8
    constexpr float CB[8] = {0.939692620785908384f, 0.766044443118978035f, 0.5f, 0.173648177666930349f,
                             -0.173648177666930349f, -0.5f, -0.766044443118978035f, -0.939692620785908384f};
    constexpr float SB[8] = {0.342020143325668733f, 0.642787609686539326f, 0.866025403784438647f,
                             0.984807753012208059f, 0.984807753012208059f, 0.866025403784438647f,
                             0.642787609686539326f, 0.342020143325668733f};
    float2 e[9], o[9];
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        e[b] = cadd(v[b], v[b + 9]);
        o[b] = csub(v[b], v[b + 9]);
    }
#pragma unroll
    for (int b = 1; b < 9; ++b) o[b] = rot<DIR>(o[b], CB[b - 1], SB[b - 1]);
    dft9<DIR>(e);
    dft9<DIR>(o);
#pragma unroll
    for (int d = 0; d < 9; ++d) {
        v[2 * d] = e[d];
        v[2 * d + 1] = o[d];
    }
}

// exp(dir 2 pi i m / 288) from the table of exp(-2 pi i m / 288) in shared memory
template <int DIR>
__device__ __forceinline__ float2 tw288(const float2* tws, int m) {
    float2 w = tws[m];
    if (DIR > 0) w.y = -w.y;
    return w;
}

}  // namespace sgw
