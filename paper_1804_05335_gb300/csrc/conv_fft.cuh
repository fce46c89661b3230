// The convolver's L-point FFT building blocks (L = 16*16*Q, T = L/16 threads,
// 16 complex values per thread), shared by the convolver and the template
// bank generator: the bank must be transformed by the same permutation-free
// forward FFT as the segments (Section 4.2).
//
// Thread/register distributions (p = position in the length-L array):
//   D1: thread t, reg i                         p = i*T + t
//   D2: thread t = a*Q + c, reg b               p = a*T + b*Q + c
//   D3: thread t = a*Q + c, reg i = s*Q + c2    p = a*T + (c + Q*s)*Q + c2
// The forward FFT is decimation in frequency: radix 16 over D1 (digit n0),
// radix 16 over D2 (n1), radix Q over D3 (n2), leaving frequency
// k = a + 16*(c + Q*s) + 256*c2 in (thread t, reg i) of D3 (digit-reversed).
// The D1 <-> D2 exchange uses rows of T+Q float2 per digit a; the D2 <-> D3
// exchange stays inside the Q-thread group of digit a, in a block of
// G = 16*(Q+1)+Q float2 with rows of Q+1.  Both layouts are free of shared
// memory bank conflicts for every access pattern used.
#pragma once
#include "dft.cuh"

namespace fdas {

template <int L>
struct ConvShape {
    static constexpr int T = L / 16;
    static constexpr int Q = L / 256;
    static constexpr int NS = 16 / Q;
    static constexpr int X1S = 16 * (T + Q);
    static constexpr int G = 16 * (Q + 1) + Q;
    static constexpr int X2S = 16 * G;
    static constexpr int BUFS = X1S > X2S ? X1S : X2S;   // float2 per exchange buffer
    // bank row: L digit-reversed slots, then 16 slots holding H[-k] for the
    // frequencies of thread 0 (see thread0_mirror), in float2
    static constexpr int ROW = L + 16;
};

// Register of thread 0 (D3) that holds -k for the frequency k of its register
// i: its 16 frequencies are closed under negation (k = 256 c2 + 16 Q s).
template <int Q>
__host__ __device__ constexpr int thread0_mirror(int i) {
    return i < Q ? (Q - i) % Q : 15 + Q - i;
}

// exp(-i 2 pi e / N), 0 <= e < N, N a power of two
__device__ __forceinline__ float2 fwd_twiddle(int e, int N) {
    float sn, cs;
    sincospif(2.0f * (float)e / (float)N, &sn, &cs);
    return make_float2(cs, -sn);
}

// Forward FFT: v holds D1 on entry, D3 (digit-reversed spectrum) on exit.
// Uses buf0 (D1->D2) and the thread's group block of buf1 (D2->D3); the
// caller guarantees both are free on entry.  Ends without a CTA barrier.
template <int L>
__device__ __forceinline__ void forward_fft_d3(float2* v, float2* buf0, float2* buf1, int t) {
    using S = ConvShape<L>;
    constexpr int T = S::T, Q = S::Q, G = S::G;
    const int a = t / Q, c = t % Q;
    dft16<-1>(v);
#pragma unroll
    for (int k0 = 1; k0 < 16; ++k0) v[k0] = cmul(v[k0], fwd_twiddle(t * k0, L));
#pragma unroll
    for (int i = 0; i < 16; ++i) buf0[i * (T + Q) + t] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = buf0[a * (T + Q) + i * Q + c];
    dft16<-1>(v);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], fwd_twiddle((c * k1) % (L / 16), L / 16));
    float2* x2 = buf1 + a * G;
#pragma unroll
    for (int i = 0; i < 16; ++i) x2[i * (Q + 1) + c] = v[i];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = x2[(c + Q * (i / Q)) * (Q + 1) + (i % Q)];
#pragma unroll
    for (int s2 = 0; s2 < S::NS; ++s2) dftq<Q, -1>(v + s2 * Q);
}

}  // namespace fdas
