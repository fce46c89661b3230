// fdas_normalise: real FFT of the series and block running-median
// normalisation (Section 3 workflow; Section 4.1 real-to-complex transform;
// DFT sign of Section 4.2).
//
// The n real samples are read as N = n/2 complex values z_m = x_2m + i x_2m+1
// and transformed by a three-pass N-point FFT, N = N1 N2 N3 (each factor a
// power of two 16..256; N3 = 48, 96 or 192 for a Bluestein length 3 * 2^m):
//   index n = n1 + N1 n2 + N1 N2 n3, frequency k = k3 + N3 k2 + N3 N2 k1;
//   pass A: length-N3 DFTs over n3, twiddle exp(-i 2 pi (n1 + N1 n2) k3 / N);
//   pass B: length-N2 DFTs over n2, twiddle exp(-i 2 pi n1 k2 / (N1 N2));
//   pass C: length-N1 DFTs over n1, written transposed to natural order.
// Each pass moves tiles of 16 lines x R points through shared memory with
// 128-byte coalesced rows and transforms each line by two register passes,
// R = R1 x 16: radix R1 over every 16th point, a twiddle, one padded
// transpose in shared memory, radix 16 (tile_dft_r).  A final kernel per
// median block forms the real spectrum
//   X_k = E_k + exp(-i 2 pi k / n) O_k,  E = (Z_k + conj Z_{N-k})/2,
//   O = (Z_k - conj Z_{N-k}) / 2i,   X_0 := 0,
// selects the lower median of |X_k|^2 in the block exactly (radix select on
// the float bit patterns) and scales the block by sqrt(ln 2 / median).
//
// A series whose length n is even but not a power of two takes the N-point
// DFT (N = n/2) by Bluestein's chirp-z identity: with c_m = exp(-i pi m^2/N),
//   Z_k = sum_m z_m exp(-i 2 pi m k / N) = c_k sum_m (z_m c_m) conj(c_{k-m}),
// a linear convolution evaluated as a circular one of length P >= 2N - 1
// (the least 2^m or 3 * 2^m) with the three-pass FFT above: A = FFT(z c), B = FFT(conj c
// placed circularly), D = FFT(conj(A B)), and Z_k = c_k conj(D_k) / P (the
// inverse by conjugation).  Each FFT's input is generated inside its first
// pass, and B, which depends only on n, can be computed once
// (fdas_bluestein_prepare) and passed to every call for that length
// (fdas_normalise_prepared).  m^2 is reduced modulo 2N in integers before the
// FP32 sine and cosine, so the chirp's phase error stays at the rounding of
// (m^2 mod 2N)/N.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "dft.cuh"
#include "internal.h"

namespace fdas {

constexpr int kFeThreads = 256;
constexpr int kTilePad = 17;   // tile row stride in float2 (16 lines + 1)

// Shared memory of a pass over lines of R points: R twiddles, then the tile
// x and its transpose buffer y of R rows each.
__host__ __device__ constexpr size_t tile_bytes(int R) {
    return (size_t)(R + 2 * R * kTilePad) * sizeof(float2);
}

__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Forward length-R DFT (R = R1*16, R1 = 1, 2, 3, 4, 6, 8, 12, 16) of the 16
// columns of tile x[r*17 + col].
// Thread (col = t % 16, j = t / 16) takes points r = j + 16 i, i < R1, does
// the radix-R1 DFT over i, multiplies output k1 by exp(-i 2 pi j k1 / R) and
// stores it at y[(16 k1 + j)*17 + col]; thread (col, k1) then does the
// radix-16 DFT over j and writes frequency k = k1 + R1 k2 to x[k*17 + col].
// Every access pattern touches each bank pair at most twice per warp.
// tw[q] = exp(-i 2 pi q / R), q < R.  Ends with a barrier; returns x.
template <int R1>
__device__ void tile_dft_r(float2* x, float2* y, const float2* tw) {
    const int t = threadIdx.x, col = t & 15, jj = t >> 4;
    float2 v[16];
    if constexpr (R1 > 1) {
#pragma unroll
        for (int i = 0; i < R1; ++i) v[i] = x[(jj + 16 * i) * kTilePad + col];
        if constexpr (R1 == 2) {
            dft2<-1>(v[0], v[1]);
        } else if constexpr (R1 == 3) {
            dft3<-1>(v[0], v[1], v[2]);
        } else if constexpr (R1 == 6) {
            dft6<-1>(v);
        } else if constexpr (R1 == 12) {
            dft12<-1>(v);
        } else if constexpr (R1 == 4) {
            dft4<-1>(v[0], v[1], v[2], v[3]);
        } else if constexpr (R1 == 8) {
            dft8<-1>(v);
        } else {
            dft16<-1>(v);
        }
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) v[k1] = c_mul(v[k1], tw[jj * k1]);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) y[(16 * k1 + jj) * kTilePad + col] = v[k1];
    } else {
        y[jj * kTilePad + col] = x[jj * kTilePad + col];
    }
    __syncthreads();
    if (jj < R1) {
        const int k1 = jj;
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = y[(16 * k1 + j) * kTilePad + col];
        dft16<-1>(v);
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) x[(k1 + R1 * k2) * kTilePad + col] = v[k2];
    }
    __syncthreads();
}

// tw[q] = exp(-i 2 pi q / R), q < R
template <int R>
__device__ __forceinline__ void load_tw(float2* tw) {
    for (int q = threadIdx.x; q < R; q += blockDim.x) {
        float s, c;
        sincospif((float)q * (2.0f / (float)R), &s, &c);
        tw[q] = make_float2(c, -s);
    }
}

// exp(-i pi x) for x = 2 e / N given as a float (e < N <= 2^24 is exact in
// float; e * (2/N) is exact for a power-of-two N and within about an ulp for
// N = 3 * 2^m; no division is needed)
__device__ __forceinline__ float2 twiddle_pi(float x) {
    float s, c;
    sincospif(x, &s, &c);
    return make_float2(c, -s);
}

// A pass over lines of R points (R = 16 .. 256, a power of two, or 48, 96,
// 192 for pass A; a compile-time constant):
// each CTA of 256 threads moves 16 lines, thread t taking column t % 16 of
// rows t / 16 + 16 s (passes A, B) or point t % R of lines t / R + (256/R) s
// (pass C), s < R/16.  All R/16 loads are issued before the first store to
// shared memory, so a thread keeps them in flight together.
template <int R>
struct FeLine {
    static constexpr int R1 = R / 16;
    static constexpr int PER = R / 16;        // values per thread
};

// Inputs of pass A: src(j) is the j-th value of the FFT's input.
struct SrcPlain {   // a stored array
    const float2* a;
    __device__ __forceinline__ float2 operator()(int64_t j) const { return __ldg(&a[j]); }
};

// pass A: DFT over n3 (length R = N3, stride N12), 16 consecutive lines m per
// CTA; output k3 of line m times exp(-i 2 pi m k3 / N) (m k3 < N)
template <int R, class Src>
__global__ void __launch_bounds__(kFeThreads) fe_pass_a(const Src src, float2* __restrict__ out,
                                                        int64_t N12, float two_over_n) {
    extern __shared__ float2 fsm[];
    float2* tw = fsm;
    float2* x = tw + R;
    float2* y = x + R * kTilePad;
    constexpr int PER = FeLine<R>::PER;
    const int t = threadIdx.x, col = t & 15, rr = t >> 4;
    const int64_t m = (int64_t)blockIdx.x * 16 + col;
    float2 ld[PER];
#pragma unroll
    for (int s = 0; s < PER; ++s) ld[s] = src(m + (int64_t)(rr + 16 * s) * N12);
    load_tw<R>(tw);
#pragma unroll
    for (int s = 0; s < PER; ++s) x[(rr + 16 * s) * kTilePad + col] = ld[s];
    __syncthreads();
    tile_dft_r<FeLine<R>::R1>(x, y, tw);
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        const int k3 = rr + 16 * s;
        out[m + k3 * N12] =
            c_mul(x[k3 * kTilePad + col], twiddle_pi((float)(m * k3) * two_over_n));
    }
}

// pass B: DFT over n2 (length R = N2, stride N1), in place; 16 consecutive
// n1 per CTA; output k2 of line n1 times exp(-i 2 pi n1 k2 / (N1 N2))
template <int R>
__global__ void __launch_bounds__(kFeThreads) fe_pass_b(float2* __restrict__ buf, int N1,
                                                        float two_over_n12) {
    extern __shared__ float2 fsm[];
    float2* tw = fsm;
    float2* x = tw + R;
    float2* y = x + R * kTilePad;
    constexpr int PER = FeLine<R>::PER;
    const int chunks = N1 / 16;
    const int t = threadIdx.x, col = t & 15, rr = t >> 4;
    const int64_t k3 = blockIdx.x / chunks;
    const int n1 = (blockIdx.x % chunks) * 16 + col;
    const int64_t base = k3 * N1 * R + n1;
    float2 ld[PER];
#pragma unroll
    for (int s = 0; s < PER; ++s) ld[s] = buf[base + (int64_t)(rr + 16 * s) * N1];
    load_tw<R>(tw);
#pragma unroll
    for (int s = 0; s < PER; ++s) x[(rr + 16 * s) * kTilePad + col] = ld[s];
    __syncthreads();
    tile_dft_r<FeLine<R>::R1>(x, y, tw);
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        const int k2 = rr + 16 * s;
        buf[base + (int64_t)k2 * N1] =
            c_mul(x[k2 * kTilePad + col], twiddle_pi((float)(n1 * k2) * two_over_n12));
    }
}

// pass C: DFT over n1 (contiguous, length R = N1); 16 consecutive k3 per CTA,
// written to natural order X[k3 + N3 k2 + N3 N2 k1]
template <int R>
__global__ void __launch_bounds__(kFeThreads) fe_pass_c(const float2* __restrict__ in,
                                                        float2* __restrict__ out, int N2, int N3) {
    extern __shared__ float2 fsm[];
    float2* tw = fsm;
    float2* x = tw + R;
    float2* y = x + R * kTilePad;
    constexpr int PER = FeLine<R>::PER;
    const int chunks = N3 / 16;
    const int64_t k2 = blockIdx.x / chunks;
    const int64_t k30 = (int64_t)(blockIdx.x % chunks) * 16;
    const int64_t N12 = (int64_t)R * N2;
    const int t = threadIdx.x, r = t % R, c0 = t / R;
    float2 ld[PER];
#pragma unroll
    for (int s = 0; s < PER; ++s)
        ld[s] = __ldg(&in[(k30 + c0 + (256 / R) * s) * N12 + k2 * R + r]);
    load_tw<R>(tw);
#pragma unroll
    for (int s = 0; s < PER; ++s) x[r * kTilePad + c0 + (256 / R) * s] = ld[s];
    __syncthreads();
    tile_dft_r<FeLine<R>::R1>(x, y, tw);
    const int64_t N32 = (int64_t)N3 * N2;
    const int col = t & 15, rr = t >> 4;
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        const int k1 = rr + 16 * s;
        out[k30 + col + N3 * k2 + N32 * k1] = x[k1 * kTilePad + col];
    }
}

// Exact rank-`rank` element of the CTA's keys (unsigned order, every key
// below 2^31: non-negative floats), KPT per thread in registers (keys past
// the block hold 0xffffffff and match no prefix), by radix select on bits
// 30-23, 22-15, 14-7, 6-0; every thread of the CTA returns it.  The
// histograms and results alternate between two buffers, so a round takes two
// barriers: the CTA counts the keys that match the prefix into hist[r & 1];
// then warp 0 scans it while the other warps clear the next round's buffer.
// hist[0] must be zero (and visible to all threads) on entry.
template <int KPT>
__device__ uint32_t radix_select(const uint32_t (&key)[KPT], int rank, uint32_t (*hist)[256],
                                 int (*bc)[2]) {
    uint32_t prefix = 0, pmask = 0;
#pragma unroll 1
    for (int round = 0; round < 4; ++round) {
        const int shift = round < 3 ? 23 - 8 * round : 0;
        const uint32_t dmask = round < 3 ? 255u : 127u;
        uint32_t* h0 = hist[round & 1];
#pragma unroll
        for (int s = 0; s < KPT; ++s)
            if ((key[s] & pmask) == prefix && key[s] != 0xffffffffu)
                atomicAdd(&h0[(key[s] >> shift) & dmask], 1u);
        __syncthreads();
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            const uint4 a = reinterpret_cast<const uint4*>(h0)[2 * l];
            const uint4 b = reinterpret_cast<const uint4*>(h0)[2 * l + 1];
            const uint32_t h[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            uint32_t sum = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) sum += h[e];
            uint32_t inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
                if (l >= o) inc += v;
            }
            const unsigned hit = __ballot_sync(0xffffffffu, inc > (uint32_t)rank);
            const int L0 = __ffs(hit) - 1;
            if (l == L0) {
                uint32_t base = inc - sum;
                int d = 0;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if (base + h[e] > (uint32_t)rank) { d = e; break; }
                    base += h[e];
                }
                bc[round & 1][0] = 8 * l + d;
                bc[round & 1][1] = rank - (int)base;
            }
        } else {
            // threads 32..255 clear bins 32..255, threads 32..63 also bins 0..31
            hist[(round + 1) & 1][threadIdx.x] = 0;
            if (threadIdx.x < 64) hist[(round + 1) & 1][threadIdx.x - 32] = 0;
        }
        __syncthreads();
        rank = bc[round & 1][1];
        prefix |= (uint32_t)bc[round & 1][0] << shift;
        pmask |= dmask << shift;
    }
    return prefix;
}

// c_m = exp(-i pi m^2 / N) for 0 <= m < N <= 2^23: r = m^2 mod 2N exactly (a
// float estimate of the quotient, within 2 of it, corrected in integers),
// then the FP32 sine and cosine of pi r / N.
__device__ __forceinline__ float2 chirp(int64_t m, int64_t N, float inv_2n, float inv_n) {
    const int64_t two_n = 2 * N, sq = m * m;
    int64_t r = sq - (int64_t)((float)sq * inv_2n) * two_n;
    while (r < 0) r += two_n;
    while (r >= two_n) r -= two_n;
    float s, c;
    sincospif((float)r * inv_n, &s, &c);
    return make_float2(c, -s);
}

// Z_k of the N-point DFT from the FFT output D: Z = D (power-of-two N) or,
// after Bluestein's convolution of length P, Z_k = c_k conj(D_k) / P.
template <bool BLUE>
__device__ __forceinline__ float2 z_value(const float2* __restrict__ D, int64_t k, int64_t N,
                                          float inv_p, float inv_2n, float inv_n) {
    const float2 d = D[k];
    if constexpr (!BLUE) {
        return d;
    } else {
        const float2 c = chirp(k, N, inv_2n, inv_n);
        return make_float2(inv_p * fmaf(c.x, d.x, c.y * d.y), inv_p * fmaf(c.y, d.x, -c.x * d.y));
    }
}

// one CTA of 256 threads per median block (at most 256 KPT bins):
// real-spectrum post-processing + normalisation.  Thread t takes bins
// k0 + t + 256 s, s < KPT, kept in registers.  inv_n = 1/N (exact for
// power-of-two N), inv_2n = 1/(2N).
template <bool BLUE, int KPT>
__global__ void __launch_bounds__(kFeThreads) fe_post(const float2* __restrict__ Z,
                                                      float2* __restrict__ spec, int64_t N,
                                                      int block, float inv_p, float inv_n,
                                                      float inv_2n) {
    __shared__ __align__(16) uint32_t hist[2][256];
    __shared__ int bc[2][2];
    const int64_t k0 = (int64_t)blockIdx.x * block;
    const int len = (int)min((int64_t)block, N - k0);
    hist[0][threadIdx.x] = 0;   // 256 threads
    float2 X[KPT];
    uint32_t key[KPT];
#pragma unroll
    for (int s = 0; s < KPT; ++s) {
        const int i = threadIdx.x + kFeThreads * s;
        X[s] = make_float2(0.f, 0.f);
        key[s] = 0xffffffffu;
        if (i < len) {
            const int64_t k = k0 + i;
            const float2 zk = z_value<BLUE>(Z, k, N, inv_p, inv_2n, inv_n);
            const float2 zm = z_value<BLUE>(Z, k == 0 ? 0 : N - k, N, inv_p, inv_2n, inv_n);
            const float ex = 0.5f * (zk.x + zm.x), ey = 0.5f * (zk.y - zm.y);
            const float ox = 0.5f * (zk.y + zm.y), oy = -0.5f * (zk.x - zm.x);
            float sn, cs;
            sincospif((float)k * inv_n, &sn, &cs);   // 2 pi k / n = pi k / N
            // w = (cs, -sn):  X = E + w O
            if (k != 0) X[s] = make_float2(ex + fmaf(cs, ox, sn * oy), ey + fmaf(cs, oy, -sn * ox));
            key[s] = __float_as_uint(fmaf(X[s].x, X[s].x, X[s].y * X[s].y));
        }
    }
    __syncthreads();
    const uint32_t mk = radix_select<KPT>(key, (len - 1) / 2, hist, bc);
    const float med = __uint_as_float(mk);
    const float scale = med > 0.f ? sqrtf(0.69314718055994531f / med) : 0.f;
#pragma unroll
    for (int s = 0; s < KPT; ++s) {
        const int i = threadIdx.x + kFeThreads * s;
        if (i < len) spec[k0 + i] = make_float2(X[s].x * scale, X[s].y * scale);
    }
}

// The post kernel for median blocks of `block` bins (32 .. 8192)
template <bool BLUE>
static int launch_post(const float2* Z, float2* spec, int64_t N, int block, float inv_p,
                       float inv_n, float inv_2n, cudaStream_t st) {
    const int nblk = (int)((N + block - 1) / block);
    const int kpt = (block + kFeThreads - 1) / kFeThreads;
    auto go = [&](auto kk) {
        constexpr int K = decltype(kk)::value;
        fe_post<BLUE, K><<<nblk, kFeThreads, 0, st>>>(Z, spec, N, block, inv_p, inv_n, inv_2n);
        return cuda_status(cudaGetLastError());
    };
    if (kpt <= 1) return go(std::integral_constant<int, 1>{});
    if (kpt <= 2) return go(std::integral_constant<int, 2>{});
    if (kpt <= 4) return go(std::integral_constant<int, 4>{});
    if (kpt <= 8) return go(std::integral_constant<int, 8>{});
    if (kpt <= 16) return go(std::integral_constant<int, 16>{});
    return go(std::integral_constant<int, 32>{});
}

// Bluestein's three FFT inputs, generated inside pass A of each FFT:
// a[m] = z_m c_m (m < N, then zeros up to P) ...
struct SrcChirpIn {
    const float2* z;
    int64_t N;
    float inv_2n, inv_n;
    __device__ __forceinline__ float2 operator()(int64_t m) const {
        return m < N ? c_mul(__ldg(&z[m]), chirp(m, N, inv_2n, inv_n)) : make_float2(0.f, 0.f);
    }
};
// ... the convolution kernel conj(c_j), j in (-N, N), placed circularly in P ...
struct SrcChirpKernel {
    int64_t N, P;
    float inv_2n, inv_n;
    __device__ __forceinline__ float2 operator()(int64_t j) const {
        const int64_t d = j < N ? j : (j > P - N ? P - j : -1);
        const float2 c = d >= 0 ? chirp(d, N, inv_2n, inv_n) : make_float2(0.f, 0.f);
        return make_float2(c.x, -c.y);
    }
};
// ... and conj(A B), the product of the two spectra conjugated, so that a
// forward FFT of it gives the conjugated inverse.
struct SrcProductConj {
    const float2* a;
    const float2* b;
    __device__ __forceinline__ float2 operator()(int64_t k) const {
        const float2 p = c_mul(a[k], b[k]);
        return make_float2(p.x, -p.y);
    }
};

static int log2i(int64_t v) {
    int p = 0;
    while (((int64_t)1 << p) < v) ++p;
    return p;
}

// Bluestein convolution length for a series of n samples (n even, not a
// power of two): the least length >= n - 1 = 2N - 1 of the form 2^m or
// 3 * 2^m (3 * 2^12 <= 3 * 2^m <= 3 * 2^22); 0 if n is out of range.
static int64_t bluestein_length(int64_t n) {
    if (n < (1 << 13) || n > ((int64_t)1 << 24) || (n & 1) || !(n & (n - 1))) return 0;
    int64_t P = 1;
    while (P < n - 1) P <<= 1;
    int64_t P3 = (int64_t)3 << 12;
    while (P3 < n - 1) P3 <<= 1;
    return (P3 < P && P3 <= ((int64_t)3 << 22)) ? P3 : P;
}

// f(std::integral_constant<int, R>) for the line length R = 16 .. 256 (powers
// of two, and 48, 96, 192 for pass A of a length 3 * 2^m)
template <class F>
static int with_line(int R, F&& f) {
    switch (R) {
        case 16: return f(std::integral_constant<int, 16>{});
        case 32: return f(std::integral_constant<int, 32>{});
        case 48: return f(std::integral_constant<int, 48>{});
        case 96: return f(std::integral_constant<int, 96>{});
        case 192: return f(std::integral_constant<int, 192>{});
        case 64: return f(std::integral_constant<int, 64>{});
        case 128: return f(std::integral_constant<int, 128>{});
        case 256: return f(std::integral_constant<int, 256>{});
        default: return FDAS_E_UNSUPPORTED;
    }
}

// The factors N = N1 N2 N3 of a transform length N = 2^m (2^12 .. 2^24) or
// 3 * 2^m (3 * 2^12 .. 3 * 2^22): powers of two between 16 and 256, except
// N3 = 3 * 2^a between 48 and 192 when 3 divides N.
static void fft_factors(int64_t N, int& N1, int& N2, int& N3) {
    const bool three = (N % 3) == 0;
    const int p = log2i(three ? N / 3 : N);
    int p3 = p / 3, p2 = (p - p3) / 2, p1 = p - p2 - p3;
    if (three) {
        while (p3 > 6) {   // the pass A line 3 * 2^p3 stays <= 192
            --p3;
            if (p1 <= p2) ++p1; else ++p2;
        }
    }
    N1 = 1 << p1;
    N2 = 1 << p2;
    N3 = (three ? 3 : 1) << p3;
}

// The three-pass forward FFT of N points (fft_factors): pass A src -> mid,
// pass B in place in mid, pass C mid -> out (natural order).
template <class Src>
static int fft3(const Src& src, float2* mid, float2* out, int64_t N, cudaStream_t st) {
    int N1, N2, N3;
    fft_factors(N, N1, N2, N3);
    const int64_t N12 = (int64_t)N1 * N2;
    // 2/N12 is exact (a power of two), 2/N too unless 3 divides N
    const float two_over_n = 2.0f / (float)N, two_over_n12 = 2.0f / (float)N12;
    int rc = with_line(N3, [&](auto r) {
        constexpr int R = decltype(r)::value;
        const int q = kernel_setup(reinterpret_cast<const void*>(&fe_pass_a<R, Src>),
                                   tile_bytes(R), kFeThreads, nullptr, nullptr, 100);
        if (q != FDAS_OK) return q;
        fe_pass_a<R, Src><<<(unsigned)(N12 / 16), kFeThreads, tile_bytes(R), st>>>(src, mid, N12,
                                                                                    two_over_n);
        return FDAS_OK;
    });
    if (rc == FDAS_OK)
        rc = with_line(N2, [&](auto r) {
            constexpr int R = decltype(r)::value;
            const int q = kernel_setup(reinterpret_cast<const void*>(&fe_pass_b<R>), tile_bytes(R),
                                       kFeThreads, nullptr, nullptr, 100);
            if (q != FDAS_OK) return q;
            fe_pass_b<R><<<(unsigned)(N3 * (N1 / 16)), kFeThreads, tile_bytes(R), st>>>(
                mid, N1, two_over_n12);
            return FDAS_OK;
        });
    if (rc == FDAS_OK)
        rc = with_line(N1, [&](auto r) {
            constexpr int R = decltype(r)::value;
            const int q = kernel_setup(reinterpret_cast<const void*>(&fe_pass_c<R>), tile_bytes(R),
                                       kFeThreads, nullptr, nullptr, 100);
            if (q != FDAS_OK) return q;
            fe_pass_c<R><<<(unsigned)(N2 * (N3 / 16)), kFeThreads, tile_bytes(R), st>>>(mid, out,
                                                                                       N2, N3);
            return FDAS_OK;
        });
    return rc != FDAS_OK ? rc : cuda_status(cudaGetLastError());
}

}  // namespace fdas

using namespace fdas;

extern "C" {

size_t fdas_normalise_workspace_bytes(int64_t n) {
    if (n >= (1 << 13) && n <= ((int64_t)1 << 25) && !(n & (n - 1)))
        return (size_t)(n / 2) * sizeof(float2);
    const int64_t P = bluestein_length(n);
    return P ? (size_t)(3 * P) * sizeof(float2) : 0;
}

size_t fdas_bluestein_bytes(int64_t n) {
    return (size_t)bluestein_length(n) * sizeof(float2);
}

int fdas_bluestein_prepare(int64_t n, void* chirp_spec, void* work, size_t work_bytes,
                           void* stream) {
    const int64_t P = bluestein_length(n);
    if (!P || !chirp_spec || !work) return FDAS_E_INVAL;
    if (work_bytes < fdas_normalise_workspace_bytes(n)) return FDAS_E_INVAL;
    if (!aligned(chirp_spec, 16) || !aligned(work, 16)) return FDAS_E_INVAL;
    const int64_t N = n / 2;
    const float inv_n = 1.0f / (float)N, inv_2n = 0.5f / (float)N;
    return fft3(SrcChirpKernel{N, P, inv_2n, inv_n}, reinterpret_cast<float2*>(work),
                reinterpret_cast<float2*>(chirp_spec), P, (cudaStream_t)stream);
}

}  // extern "C"

namespace fdas {
// fdas_normalise (chirp_spec NULL: the Bluestein kernel spectrum computed
// here) and fdas_normalise_prepared (supplied)
static int normalise_impl(const float* series, int64_t n, int32_t median_block, float* spec,
                          void* work, size_t work_bytes, const void* chirp_spec, void* stream) {
    if (!series || !spec || !work) return FDAS_E_INVAL;
    const size_t need = fdas_normalise_workspace_bytes(n);
    if (need == 0 || work_bytes < need) return FDAS_E_INVAL;
    if (median_block < 32 || median_block > 8192) return FDAS_E_INVAL;
    if (!aligned(series, 8) || !aligned(spec, 8) || !aligned(work, 16)) return FDAS_E_INVAL;
    const bool pow2 = !(n & (n - 1));
    if (!pow2 && chirp_spec && !aligned(chirp_spec, 16)) return FDAS_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = n / 2;
    int rc = FDAS_OK;
    float2* sp = reinterpret_cast<float2*>(spec);
    float2* wk = reinterpret_cast<float2*>(work);
    const float2* z = reinterpret_cast<const float2*>(series);
    const float inv_n = 1.0f / (float)N, inv_2n = 0.5f / (float)N;
    if (pow2) {
        // power of two: the N-point FFT through the spectrum buffer into the workspace
        if ((rc = fft3(SrcPlain{z}, sp, wk, N, st)) != FDAS_OK) return rc;
        return launch_post<false>(wk, sp, N, median_block, 1.f, inv_n, inv_2n, st);
    }
    // Bluestein: workspace = [X | Bk | tmp], P complex each; each FFT's input
    // is generated in its first pass; Bk only when no prepared spectrum is given
    const int64_t P = bluestein_length(n);
    float2* X = wk;
    float2* Bk = wk + P;
    float2* tmp = wk + 2 * P;
    if ((rc = fft3(SrcChirpIn{z, N, inv_2n, inv_n}, tmp, X, P, st)) != FDAS_OK) return rc;
    const float2* B = reinterpret_cast<const float2*>(chirp_spec);
    if (!B) {
        if ((rc = fft3(SrcChirpKernel{N, P, inv_2n, inv_n}, tmp, Bk, P, st)) != FDAS_OK) return rc;
        B = Bk;
    }
    if ((rc = fft3(SrcProductConj{X, B}, tmp, X, P, st)) != FDAS_OK) return rc;
    return launch_post<true>(X, sp, N, median_block, 1.0f / (float)P, inv_n, inv_2n, st);
}
}  // namespace fdas

extern "C" {

int fdas_normalise_prepared(const float* series, int64_t n, int32_t median_block, float* spec,
                            void* work, size_t work_bytes, const void* chirp_spec,
                            void* stream) {
    if ((n & (n - 1)) && !chirp_spec) return FDAS_E_INVAL;
    return normalise_impl(series, n, median_block, spec, work, work_bytes, chirp_spec, stream);
}

int fdas_normalise(const float* series, int64_t n, int32_t median_block, float* spec, void* work,
                   size_t work_bytes, void* stream) {
    return normalise_impl(series, n, median_block, spec, work, work_bytes, nullptr, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// fdas_normalise_noalloc: fdas_normalise with the workspace taken from a
// fixed device array of this file instead of the caller (for callers that
// must not allocate device memory when they call in).
// ---------------------------------------------------------------------------
namespace fdas {

constexpr size_t kNoallocScratchBytes = (size_t)(FDAS_NOALLOC_MAX_N / 2) * sizeof(float2);
static __device__ __align__(256) float2 g_noalloc_scratch[FDAS_NOALLOC_MAX_N / 2];

constexpr int kMaxDevices = 64;
static void* g_noalloc_ptr[kMaxDevices];
static std::mutex g_noalloc_mutex;

// Device address of this device's copy of the array (looked up once per
// device, with that device current).  In host code the array's name is only
// a host-side handle, never a device address.
static int noalloc_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FDAS_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FDAS_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FDAS_E_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return FDAS_OK;
}

}  // namespace fdas

extern "C" int fdas_normalise_noalloc(const float* series, int64_t n, int32_t median_block,
                                      float* spec, void* stream) {
    if (n > FDAS_NOALLOC_MAX_N || (n > 0 && (n & (n - 1)))) return FDAS_E_UNSUPPORTED;
    const size_t need = fdas_normalise_workspace_bytes(n);
    if (need == 0 || need > fdas::kNoallocScratchBytes) return FDAS_E_INVAL;
    void* work = nullptr;
    const int rc = fdas::noalloc_scratch(&work);
    if (rc != FDAS_OK) return rc;
    return fdas_normalise(series, n, median_block, spec, work, fdas::kNoallocScratchBytes, stream);
}
