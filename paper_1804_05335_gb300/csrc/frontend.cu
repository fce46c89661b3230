// fdas_normalise: real FFT of the series and block running-median
// normalisation (Section 3 workflow; Section 4.1 real-to-complex transform;
// DFT sign of Section 4.2).
//
// The n real samples are read as N = n/2 complex values z_m = x_2m + i x_2m+1
// and transformed by a three-pass N-point FFT, N = N1 N2 N3 (each factor
// 16..256):
//   index n = n1 + N1 n2 + N1 N2 n3, frequency k = k3 + N3 k2 + N3 N2 k1;
//   pass A: length-N3 DFTs over n3, twiddle exp(-i 2 pi (n1 + N1 n2) k3 / N);
//   pass B: length-N2 DFTs over n2, twiddle exp(-i 2 pi n1 k2 / (N1 N2));
//   pass C: length-N1 DFTs over n1, written transposed to natural order.
// Each pass moves tiles of 16 lines x R points through shared memory with
// 128-byte coalesced rows and transforms each line by two register passes,
// R = R1 x 16: radix R1 over every 16th point, a twiddle, one padded
// transpose in shared memory, radix 16 (tile_dft).  A final kernel per median block forms the real spectrum
//   X_k = E_k + exp(-i 2 pi k / n) O_k,  E = (Z_k + conj Z_{N-k})/2,
//   O = (Z_k - conj Z_{N-k}) / 2i,   X_0 := 0,
// selects the lower median of |X_k|^2 in the block exactly (radix select on
// the float bit patterns) and scales the block by sqrt(ln 2 / median).
//
// A series whose length n is even but not a power of two takes the N-point
// DFT (N = n/2) by Bluestein's chirp-z identity: with c_m = exp(-i pi m^2/N),
//   Z_k = sum_m z_m exp(-i 2 pi m k / N) = c_k sum_m (z_m c_m) conj(c_{k-m}),
// a linear convolution evaluated as a circular one of power-of-two length
// P >= 2N - 1 with the three-pass FFT above: A = FFT(z c), B = FFT(conj c
// placed circularly), D = FFT(conj(A B)), and Z_k = c_k conj(D_k) / P (the
// inverse by conjugation).  m^2 is reduced modulo 2N in integers before the
// FP32 sine and cosine, so the chirp's phase error stays at the rounding of
// (m^2 mod 2N)/N.
#include <math.h>

#include <algorithm>
#include <mutex>

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

// Forward length-R DFT (R = R1*16) of the 16 columns of tile x[r*17 + col].
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

__device__ float2* tile_dft(float2* x, float2* y, const float2* tw, int R) {
    switch (R) {
        case 16: tile_dft_r<1>(x, y, tw); break;
        case 32: tile_dft_r<2>(x, y, tw); break;
        case 64: tile_dft_r<4>(x, y, tw); break;
        case 128: tile_dft_r<8>(x, y, tw); break;
        default: tile_dft_r<16>(x, y, tw); break;
    }
    return x;
}

__device__ void load_tw(float2* tw, int R) {
    for (int q = threadIdx.x; q < R; q += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)q / (float)R, &s, &c);
        tw[q] = make_float2(c, -s);
    }
}

// exp(-i 2 pi e / N) with 0 <= e < N (N a power of two, e exact in float)
__device__ __forceinline__ float2 twiddle(int64_t e, int64_t N) {
    float s, c;
    sincospif(2.0f * (float)e / (float)N, &s, &c);
    return make_float2(c, -s);
}

// pass A: DFT over n3 (length N3, stride N12), 16 consecutive lines m per CTA
__global__ void __launch_bounds__(kFeThreads) fe_pass_a(const float2* __restrict__ in,
                                                        float2* __restrict__ out, int N3,
                                                        int64_t N12, int64_t N) {
    extern __shared__ float2 fsm[];
    float2* tw = fsm;
    float2* x = tw + N3;
    float2* y = x + N3 * kTilePad;
    const int64_t m0 = (int64_t)blockIdx.x * 16;
    load_tw(tw, N3);
    for (int idx = threadIdx.x; idx < 16 * N3; idx += blockDim.x) {
        const int col = idx & 15, r = idx >> 4;
        x[r * kTilePad + col] = in[m0 + col + r * N12];
    }
    __syncthreads();
    float2* res = tile_dft(x, y, tw, N3);
    for (int idx = threadIdx.x; idx < 16 * N3; idx += blockDim.x) {
        const int col = idx & 15, k3 = idx >> 4;
        const int64_t m = m0 + col;
        out[m + k3 * N12] = c_mul(res[k3 * kTilePad + col], twiddle((m * k3) % N, N));
    }
}

// pass B: DFT over n2 (length N2, stride N1), in place; 16 consecutive n1 per CTA
__global__ void __launch_bounds__(kFeThreads) fe_pass_b(float2* __restrict__ buf, int N1, int N2) {
    extern __shared__ float2 fsm[];
    float2* tw = fsm;
    float2* x = tw + N2;
    float2* y = x + N2 * kTilePad;
    const int chunks = N1 / 16;
    const int64_t k3 = blockIdx.x / chunks;
    const int n10 = (blockIdx.x % chunks) * 16;
    const int64_t N12 = (int64_t)N1 * N2;
    const int64_t base = k3 * N12 + n10;
    load_tw(tw, N2);
    for (int idx = threadIdx.x; idx < 16 * N2; idx += blockDim.x) {
        const int col = idx & 15, r = idx >> 4;
        x[r * kTilePad + col] = buf[base + col + (int64_t)r * N1];
    }
    __syncthreads();
    float2* res = tile_dft(x, y, tw, N2);
    for (int idx = threadIdx.x; idx < 16 * N2; idx += blockDim.x) {
        const int col = idx & 15, k2 = idx >> 4;
        const int64_t e = ((int64_t)(n10 + col) * k2) % N12;
        buf[base + col + (int64_t)k2 * N1] = c_mul(res[k2 * kTilePad + col], twiddle(e, N12));
    }
}

// pass C: DFT over n1 (contiguous, length N1); 16 consecutive k3 per CTA,
// written to natural order X[k3 + N3 k2 + N3 N2 k1]
__global__ void __launch_bounds__(kFeThreads) fe_pass_c(const float2* __restrict__ in,
                                                        float2* __restrict__ out, int N1, int N2,
                                                        int N3) {
    extern __shared__ float2 fsm[];
    float2* tw = fsm;
    float2* x = tw + N1;
    float2* y = x + N1 * kTilePad;
    const int chunks = N3 / 16;
    const int64_t k2 = blockIdx.x / chunks;
    const int64_t k30 = (int64_t)(blockIdx.x % chunks) * 16;
    const int64_t N12 = (int64_t)N1 * N2;
    load_tw(tw, N1);
    for (int idx = threadIdx.x; idx < 16 * N1; idx += blockDim.x) {
        const int r = idx % N1, col = idx / N1;
        x[r * kTilePad + col] = in[(k30 + col) * N12 + k2 * N1 + r];
    }
    __syncthreads();
    float2* res = tile_dft(x, y, tw, N1);
    const int64_t N32 = (int64_t)N3 * N2;
    for (int idx = threadIdx.x; idx < 16 * N1; idx += blockDim.x) {
        const int col = idx & 15, k1 = idx >> 4;
        out[k30 + col + N3 * k2 + N32 * k1] = res[k1 * kTilePad + col];
    }
}

// Exact rank-`rank` element of keys[0..len) (unsigned order) by 8-bit radix
// select; every thread of the CTA returns it.
__device__ uint32_t radix_select(const uint32_t* keys, int len, int rank, uint32_t* hist,
                                 int* bc) {
    uint32_t prefix = 0, pmask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            const uint32_t k = keys[i];
            if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            uint32_t h[8], sum = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) { h[e] = hist[8 * l + e]; sum += h[e]; }
            uint32_t inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
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
                bc[0] = 8 * l + d;
                bc[1] = rank - (int)base;
            }
        }
        __syncthreads();
        const uint32_t dig = (uint32_t)bc[0];
        rank = bc[1];
        prefix |= dig << shift;
        pmask |= 255u << shift;
        __syncthreads();
    }
    return prefix;
}

// c_m = exp(-i pi m^2 / N) for 0 <= m < 2^24: m^2 mod 2N in integers, then FP32
__device__ __forceinline__ float2 chirp(int64_t m, int64_t N) {
    const int64_t r = (m * m) % (2 * N);
    float s, c;
    sincospif((float)r / (float)N, &s, &c);
    return make_float2(c, -s);
}

// Z_k of the N-point DFT from the FFT output D: Z = D (power-of-two N) or,
// after Bluestein's convolution of length P, Z_k = c_k conj(D_k) / P.
template <bool BLUE>
__device__ __forceinline__ float2 z_value(const float2* __restrict__ D, int64_t k, int64_t N,
                                          float inv_p) {
    const float2 d = D[k];
    if constexpr (!BLUE) {
        return d;
    } else {
        const float2 c = chirp(k, N);
        return make_float2(inv_p * fmaf(c.x, d.x, c.y * d.y), inv_p * fmaf(c.y, d.x, -c.x * d.y));
    }
}

// one CTA per median block: real-spectrum post-processing + normalisation
template <bool BLUE>
__global__ void __launch_bounds__(kFeThreads) fe_post(const float2* __restrict__ Z,
                                                      float2* __restrict__ spec, int64_t N,
                                                      int block, float inv_p) {
    extern __shared__ float2 psm[];
    float2* xs = psm;
    uint32_t* keys = reinterpret_cast<uint32_t*>(xs + block);
    __shared__ uint32_t hist[256];
    __shared__ int bc[2];
    const int64_t k0 = (int64_t)blockIdx.x * block;
    const int len = (int)min((int64_t)block, N - k0);
    const int64_t n = 2 * N;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const int64_t k = k0 + i;
        const float2 zk = z_value<BLUE>(Z, k, N, inv_p);
        const float2 zm = z_value<BLUE>(Z, k == 0 ? 0 : N - k, N, inv_p);
        const float ex = 0.5f * (zk.x + zm.x), ey = 0.5f * (zk.y - zm.y);
        const float ox = 0.5f * (zk.y + zm.y), oy = -0.5f * (zk.x - zm.x);
        float s, c;
        sincospif(2.0f * (float)k / (float)n, &s, &c);
        // w = (c, -s):  X = E + w O
        float2 X = make_float2(ex + fmaf(c, ox, s * oy), ey + fmaf(c, oy, -s * ox));
        if (k == 0) X = make_float2(0.f, 0.f);
        xs[i] = X;
        keys[i] = __float_as_uint(fmaf(X.x, X.x, X.y * X.y));
    }
    __syncthreads();
    const uint32_t mk = radix_select(keys, len, (len - 1) / 2, hist, bc);
    const float med = __uint_as_float(mk);
    const float scale = med > 0.f ? sqrtf(0.69314718055994531f / med) : 0.f;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const float2 X = xs[i];
        spec[k0 + i] = make_float2(X.x * scale, X.y * scale);
    }
}

// Bluestein inputs: a[m] = z_m c_m for m < N, 0 up to P
__global__ void __launch_bounds__(kFeThreads) bs_chirp_in(const float2* __restrict__ z,
                                                          float2* __restrict__ a, int64_t N,
                                                          int64_t P) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < P;
         m += (int64_t)gridDim.x * blockDim.x)
        a[m] = m < N ? c_mul(z[m], chirp(m, N)) : make_float2(0.f, 0.f);
}

// the convolution kernel conj(c_j), j in (-N, N), placed circularly in P
__global__ void __launch_bounds__(kFeThreads) bs_chirp_kernel(float2* __restrict__ b, int64_t N,
                                                              int64_t P) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = j < N ? j : (j > P - N ? P - j : -1);
        const float2 c = d >= 0 ? chirp(d, N) : make_float2(0.f, 0.f);
        b[j] = make_float2(c.x, -c.y);
    }
}

// x = conj(x y): the product of the two spectra, conjugated so that a forward
// FFT of it gives the conjugated inverse
__global__ void __launch_bounds__(kFeThreads) bs_mul_conj(float2* __restrict__ x,
                                                          const float2* __restrict__ y,
                                                          int64_t P) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < P;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = c_mul(x[k], y[k]);
        x[k] = make_float2(p.x, -p.y);
    }
}

static int log2i(int64_t v) {
    int p = 0;
    while (((int64_t)1 << p) < v) ++p;
    return p;
}

// Bluestein convolution length for a series of n samples (n even, not a
// power of two): the least power of two >= n - 1 = 2N - 1; 0 if out of range.
static int64_t bluestein_length(int64_t n) {
    if (n < (1 << 13) || n > ((int64_t)1 << 24) || (n & 1) || !(n & (n - 1))) return 0;
    int64_t P = 1;
    while (P < n - 1) P <<= 1;
    return P;
}

// The three-pass forward FFT of P points (a power of two, 2^12..2^24): in ->
// out (natural order; out may be in), tmp holds P values in between.
static int fft_pow2(const float2* in, float2* tmp, float2* out, int64_t P, cudaStream_t st) {
    const int p = log2i(P);
    const int p3 = p / 3, p2 = (p - p3) / 2, p1 = p - p2 - p3;
    const int N1 = 1 << p1, N2 = 1 << p2, N3 = 1 << p3;
    const int64_t N12 = (int64_t)N1 * N2;
    fe_pass_a<<<(unsigned)(N12 / 16), kFeThreads, tile_bytes(N3), st>>>(in, tmp, N3, N12, P);
    fe_pass_b<<<(unsigned)(N3 * (N1 / 16)), kFeThreads, tile_bytes(N2), st>>>(tmp, N1, N2);
    fe_pass_c<<<(unsigned)(N2 * (N3 / 16)), kFeThreads, tile_bytes(N1), st>>>(tmp, out, N1, N2,
                                                                             N3);
    return cuda_status(cudaGetLastError());
}

static int frontend_setup() {
    const size_t tile_sm = tile_bytes(256);   // the largest line (attribute)
    const size_t post_max = 8192 * (sizeof(float2) + sizeof(uint32_t));
    int rc = kernel_setup(reinterpret_cast<const void*>(&fe_pass_a), tile_sm, kFeThreads, nullptr,
                          nullptr);
    if (rc == FDAS_OK)
        rc = kernel_setup(reinterpret_cast<const void*>(&fe_pass_b), tile_sm, kFeThreads, nullptr,
                          nullptr);
    if (rc == FDAS_OK)
        rc = kernel_setup(reinterpret_cast<const void*>(&fe_pass_c), tile_sm, kFeThreads, nullptr,
                          nullptr);
    if (rc == FDAS_OK)
        rc = kernel_setup(reinterpret_cast<const void*>(&fe_post<false>), post_max, kFeThreads,
                          nullptr, nullptr);
    if (rc == FDAS_OK)
        rc = kernel_setup(reinterpret_cast<const void*>(&fe_post<true>), post_max, kFeThreads,
                          nullptr, nullptr);
    return rc;
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

int fdas_normalise(const float* series, int64_t n, int32_t median_block, float* spec, void* work,
                   size_t work_bytes, void* stream) {
    if (!series || !spec || !work) return FDAS_E_INVAL;
    const size_t need = fdas_normalise_workspace_bytes(n);
    if (need == 0 || work_bytes < need) return FDAS_E_INVAL;
    if (median_block < 32 || median_block > 8192) return FDAS_E_INVAL;
    if (!aligned(series, 8) || !aligned(spec, 8) || !aligned(work, 16)) return FDAS_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = n / 2;
    int rc = frontend_setup();
    if (rc != FDAS_OK) return rc;
    float2* sp = reinterpret_cast<float2*>(spec);
    float2* wk = reinterpret_cast<float2*>(work);
    const float2* z = reinterpret_cast<const float2*>(series);
    const int nblk = (int)((N + median_block - 1) / median_block);
    const size_t post_sm = (size_t)median_block * (sizeof(float2) + sizeof(uint32_t));
    if (!(n & (n - 1))) {
        // power of two: the N-point FFT through the spectrum buffer into the workspace
        const int p = log2i(N);
        const int p3 = p / 3, p2 = (p - p3) / 2, p1 = p - p2 - p3;
        const int N1 = 1 << p1, N2 = 1 << p2, N3 = 1 << p3;
        const int64_t N12 = (int64_t)N1 * N2;
        fe_pass_a<<<(unsigned)(N12 / 16), kFeThreads, tile_bytes(N3), st>>>(z, sp, N3, N12, N);
        fe_pass_b<<<(unsigned)(N3 * (N1 / 16)), kFeThreads, tile_bytes(N2), st>>>(sp, N1, N2);
        fe_pass_c<<<(unsigned)(N2 * (N3 / 16)), kFeThreads, tile_bytes(N1), st>>>(sp, wk, N1, N2,
                                                                                 N3);
        fe_post<false><<<nblk, kFeThreads, post_sm, st>>>(wk, sp, N, median_block, 1.f);
        return cuda_status(cudaGetLastError());
    }
    // Bluestein: workspace = [X | Bk | tmp], P complex each
    const int64_t P = bluestein_length(n);
    float2* X = wk;
    float2* Bk = wk + P;
    float2* tmp = wk + 2 * P;
    const unsigned grid = (unsigned)std::min<int64_t>((P + kFeThreads - 1) / kFeThreads, 152 * 16);
    bs_chirp_in<<<grid, kFeThreads, 0, st>>>(z, X, N, P);
    bs_chirp_kernel<<<grid, kFeThreads, 0, st>>>(Bk, N, P);
    if ((rc = cuda_status(cudaGetLastError())) != FDAS_OK) return rc;
    if ((rc = fft_pow2(X, tmp, X, P, st)) != FDAS_OK) return rc;
    if ((rc = fft_pow2(Bk, tmp, Bk, P, st)) != FDAS_OK) return rc;
    bs_mul_conj<<<grid, kFeThreads, 0, st>>>(X, Bk, P);
    if ((rc = cuda_status(cudaGetLastError())) != FDAS_OK) return rc;
    if ((rc = fft_pow2(X, tmp, X, P, st)) != FDAS_OK) return rc;
    fe_post<true><<<nblk, kFeThreads, post_sm, st>>>(X, sp, N, median_block, 1.0f / (float)P);
    return cuda_status(cudaGetLastError());
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
