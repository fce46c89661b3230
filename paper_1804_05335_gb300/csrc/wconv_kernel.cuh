// The L = 1024 overlap-save convolver: one warp per segment FFT (Sections 3,
// 4.1, 4.2).
//
// A CTA of NW warps takes a contiguous, statically balanced range of work
// units in the order (series, template group, template chunk, quad,
// template): a unit is one template applied to the quad's NW consecutive
// segments, one per warp (the chunk is the whole group unless a batched
// launch asks for fewer templates per block).
// When the quad changes, each warp loads its segment -- L bins starting at
// s*B - M/2, zero outside the spectrum -- and runs the forward FFT once
// (wfft.cuh), keeping the spectrum Y in registers.  Per unit, each warp
// multiplies Y by the template spectrum, runs the inverse FFT, forms full-
// and half-bin powers of its B useful positions and writes them to the plane.
// The whole transform stays inside the warp: one exchange through the warp's
// shared memory, no CTA barrier.
//
// Template rows are staged by bulk copies (cp.async.bulk) into NBUF shared
// buffers, each read by all four warps: one thread issues the copies in the
// order the units need them, a `full` mbarrier per buffer completes on the
// copy's bytes, and an `empty` mbarrier per buffer collects one arrival per
// warp when the warp is done with the row.  A symmetric grid pairs +z and -z
// in consecutive units on one row (H_{-z}[k] = conj(H_z[-k]), Section 4.2):
// -k of lane l, register i is lane 32 - l, register 31 - i (l >= 1); lane 0's
// values at -k sit in the row's mirror column, so every lane reads the
// conjugate row at 527 - 33 j - l.
//
// Epilogue: position p = l + 32 i of register i; the half bin needs x[p + 1],
// which lane l + 1 holds in the same register, passed by one shuffle per
// component.  Lane 31's neighbour is lane 0's next register, so lane 0
// supplies that one instead (32 lanes in a cycle cannot all find p + 1 in
// the same register of the next lane).  Each warp store covers 32
// consecutive bins (256 contiguous bytes with interbinning).
//
// Every wait is bounded.  A wait that runs out (or `A.probe` set, which arms
// the first row's barrier without issuing its copy -- a diagnostic that makes
// the wait run out with nothing in flight) sets FDAS_STATUS_TIMEOUT, stops
// every warp of the CTA through a shared flag, and the copy-issuing thread
// waits, again bounded, for its copies still in flight before the CTA exits.
#pragma once
#include "conv_common.cuh"
#include "tc_dft.cuh"
#include "tma.cuh"
#include "wfft.cuh"

namespace fdas {

template <int PREC = 0>
struct WSmem {
    static constexpr size_t base =
        (size_t)WShape::NBUF * WShape::ROW4 * sizeof(float4) +     // staged bank rows
        (size_t)WShape::TW4 * sizeof(float4) +                       // twiddle table
        (size_t)WShape::NW * WShape::XBUF * sizeof(float2);          // per-warp exchange
    // tensor-core forms: the DFT matrix parts (tc_dft.cuh)
    static constexpr size_t bytes = base + (PREC ? (size_t)TcShape<PREC ? PREC : 1>::BBYTES : 0);
};

template <int I>
struct Ic {
    static constexpr int value = I;
};
// f(Ic<I>{}) for I = I0 .. I1 - 1, unrolled at compile time
template <int I0, int I1, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I0 < I1) {
        f(Ic<I0>{});
        static_for<I0 + 1, I1>(f);
    }
}

// The series of the unit being processed: a single-series launch reads it
// from the launch arguments (no registers held), a batched launch from the
// trial table.
template <bool BATCH>
struct WSeries {
    __device__ __forceinline__ void set(const ConvArgs&, int) {}
    __device__ __forceinline__ const float2* spec(const ConvArgs& A) const { return A.spec; }
    __device__ __forceinline__ int64_t nb(const ConvArgs& A) const { return A.nb; }
    __device__ __forceinline__ float* plane(const ConvArgs& A) const { return A.plane; }
    __device__ __forceinline__ int64_t row_stride(const ConvArgs& A) const { return A.row_stride; }
    __device__ __forceinline__ int64_t end(const ConvArgs& A) const { return A.items; }
    __device__ __forceinline__ int flags() const { return 0; }
    __device__ __forceinline__ int trial() const { return 0; }
};
// (only the trial index and its last unit stay in registers; the other
// fields are read from the trial table, an L1 hit, where they are used)
template <>
struct WSeries<true> {
    int tr;
    int64_t last;   // first unit of the next trial
    __device__ __forceinline__ void set(const ConvArgs& A, int t) {
        tr = t;
        last = (t + 1 < A.ntrials) ? A.trials[t + 1].item_begin : A.items;
    }
    __device__ __forceinline__ const float2* spec(const ConvArgs& A) const {
        return reinterpret_cast<const float2*>(A.trials[tr].spec);
    }
    __device__ __forceinline__ int64_t nb(const ConvArgs& A) const { return A.trials[tr].nb; }
    __device__ __forceinline__ float* plane(const ConvArgs& A) const { return A.trials[tr].plane; }
    __device__ __forceinline__ int64_t row_stride(const ConvArgs& A) const {
        return A.trials[tr].row_stride;
    }
    __device__ __forceinline__ int64_t end(const ConvArgs&) const { return last; }
    __device__ __forceinline__ int flags() const { return tr << 8; }
    __device__ __forceinline__ int trial() const { return tr; }
};

// Walk over the work units of a series (or of a batch of series).  Within a
// template group the units run (template chunk, quad, template): A.tpb > 0
// splits the group's templates into chunks of A.tpb, each applied to every
// quad before the next chunk (templates per CTA visit of a segment); A.tpb =
// 0 keeps the whole group as one chunk, so each quad's forward FFT serves
// all of the group's templates.
template <bool BATCH, int SUB>
struct WWalk {
    int u;            // unit index
    WSeries<BATCH> ser;
    int nq;           // quads of group grp in the current series
    int quad;         // segments NW quad .. NW quad + NW - 1 of group grp
    int grp;
    int q;            // template of group grp
    int c0, cn;       // current chunk: templates c0 .. c0 + cn - 1

    __device__ __forceinline__ int64_t npos(const ConvArgs& A) const { return SUB * ser.nb(A); }
    __device__ __forceinline__ int quads(const ConvArgs& A, int g) const {
        const int64_t B = WShape::L - A.gM[g];
        return (int)(((npos(A) + B - 1) / B + WShape::NW - 1) / WShape::NW);
    }
    __device__ __forceinline__ static int chunk(const ConvArgs& A, int g) {
        return (A.tpb > 0 && A.tpb < A.gK[g]) ? A.tpb : A.gK[g];
    }
    __device__ __forceinline__ void init(const ConvArgs& A, int u0) {
        u = u0;
        int trial = 0;
        if constexpr (BATCH) {   // last trial whose first unit is <= u0
            int a0 = 0, a1 = A.ntrials - 1;
            while (a0 < a1) {
                const int mid = (a0 + a1 + 1) >> 1;
                if (A.trials[mid].item_begin <= u0) a0 = mid; else a1 = mid - 1;
            }
            trial = a0;
        }
        ser.set(A, trial);
        int64_t rel = u0 - (BATCH ? A.trials[trial].item_begin : 0);
        grp = 0;
        nq = quads(A, 0);
        while (rel >= (int64_t)nq * A.gK[grp] && grp + 1 < A.ng) {
            rel -= (int64_t)nq * A.gK[grp];
            ++grp;
            nq = quads(A, grp);
        }
        const int C = chunk(A, grp);
        c0 = (int)min(rel / ((int64_t)nq * C), (int64_t)((A.gK[grp] - 1) / C)) * C;
        cn = min(C, A.gK[grp] - c0);
        rel -= (int64_t)nq * c0;
        quad = (int)(rel / cn);
        q = c0 + (int)(rel - (int64_t)quad * cn);
    }
    // next unit; returns true if it starts a new quad (new segments)
    __device__ __forceinline__ bool advance(const ConvArgs& A) {
        ++u;
        bool fresh = false;
        if (++q == c0 + cn) {
            q = c0;
            fresh = true;
            if (++quad == nq) {
                quad = 0;
                c0 += cn;
                if (c0 == A.gK[grp]) {
                    c0 = 0;
                    if (++grp == A.ng) grp = 0;
                    nq = quads(A, grp);
                }
                cn = min(chunk(A, grp), A.gK[grp] - c0);
                q = c0;
            }
        }
        if constexpr (BATCH) {
            if (u == ser.end(A) && u < A.items) {
                ser.set(A, ser.trial() + 1);
                grp = 0;
                quad = 0;
                c0 = 0;
                cn = chunk(A, 0);
                q = 0;
                nq = quads(A, 0);
                fresh = true;
            }
        }
        return fresh;
    }
};

template <bool BATCH, int SUB>
struct WProducer {            // state of the copy-issuing thread, in shared memory
    WWalk<BATCH, SUB> walk;   // first unit whose row is not yet issued
    uint32_t issued;          // rows issued so far
};

// Bounded wait on phase `parity` of `bar`; gives up early when `abort` is set.
__device__ __forceinline__ bool wwait(uint64_t* bar, uint32_t parity, const volatile int* abort,
                                      uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 16-bit or float plane stores of one or two consecutive elements (elements
// of type OUT; the two-element store needs 2-element alignment).
template <int OUT>
__device__ __forceinline__ void wstore2(void* row, int64_t i, float a, float b) {
    if constexpr (OUT == 0) {
        __stcs(reinterpret_cast<float2*>(static_cast<float*>(row) + i), make_float2(a, b));
    } else {
        uint32_t u;
        if constexpr (OUT == 1) {
            __half2 h = __floats2half2_rn(a, b);
            u = *reinterpret_cast<uint32_t*>(&h);
        } else {
            __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            u = *reinterpret_cast<uint32_t*>(&h);
        }
        __stcs(reinterpret_cast<unsigned int*>(static_cast<uint16_t*>(row) + i), u);
    }
}
// The same stores, issued only where `ok` (one predicated instruction, no
// branch): for the registers at a segment's edges.
template <int OUT>
__device__ __forceinline__ void wstore2_if(bool ok, void* row, int64_t i, float a, float b) {
    if constexpr (OUT == 0) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t"
                     "@p st.global.cs.v2.f32 [%1], {%2, %3};\n\t}"
                     ::"r"((int)ok), "l"(static_cast<float*>(row) + i), "f"(a), "f"(b) : "memory");
    } else {
        uint32_t u;
        if constexpr (OUT == 1) {
            __half2 h = __floats2half2_rn(a, b);
            u = *reinterpret_cast<uint32_t*>(&h);
        } else {
            __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            u = *reinterpret_cast<uint32_t*>(&h);
        }
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t"
                     "@p st.global.cs.b32 [%1], %2;\n\t}"
                     ::"r"((int)ok), "l"(static_cast<uint16_t*>(row) + i), "r"(u) : "memory");
    }
}
template <int OUT>
__device__ __forceinline__ void wstore1_if(bool ok, void* row, int64_t i, float a) {
    if constexpr (OUT == 0) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t"
                     "@p st.global.cs.f32 [%1], %2;\n\t}"
                     ::"r"((int)ok), "l"(static_cast<float*>(row) + i), "f"(a) : "memory");
    } else {
        uint16_t u;
        if constexpr (OUT == 1) {
            __half h = __float2half_rn(a);
            u = *reinterpret_cast<uint16_t*>(&h);
        } else {
            __nv_bfloat16 h = __float2bfloat16_rn(a);
            u = *reinterpret_cast<uint16_t*>(&h);
        }
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t"
                     "@p st.global.cs.b16 [%1], %2;\n\t}"
                     ::"r"((int)ok), "l"(static_cast<uint16_t*>(row) + i), "h"(u) : "memory");
    }
}
template <int OUT>
__device__ __forceinline__ void wstore1(void* row, int64_t i, float a) {
    if constexpr (OUT == 0) {
        __stcs(static_cast<float*>(row) + i, a);
    } else if constexpr (OUT == 1) {
        reinterpret_cast<__half*>(row)[i] = __float2half_rn(a);
    } else {
        reinterpret_cast<__nv_bfloat16*>(row)[i] = __float2bfloat16_rn(a);
    }
}

constexpr float kHalfBinScale = 0.61685027506808491f;   // (pi/4)^2 of Eq. f-interp

// Powers of the 32 registers of one lane after wfft_inverse, for a segment
// that lies inside the series with M/2 <= 160: registers 5..26 always hold
// useful positions; the lane's useful registers are ilo .. ihi - 1 (ilo <= 5,
// ihi >= 27).  IB: full bin and interbinned half bin per position (x[p + 1]
// from lane l + 1, same register), else the full bin.  rb: the bin of
// register 0.  Returns the lane's largest power.
template <int OUT, bool IB>
__device__ __forceinline__ float wepi_fast(const float2* v, int l, int ilo, int ihi, void* prow,
                                           int64_t rb) {
    float mx = 0.f;
    static_for<0, 32>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        bool ok;
        if constexpr (i >= 5 && i <= 26) ok = true;
        else if constexpr (i < 5) ok = i >= ilo;
        else ok = i < ihi;
        const float2 x = v[i];
        const float pf = fmaf(x.x, x.x, x.y * x.y);
        if constexpr (IB) {
            const float2 pv = (l == 0) ? v[(i + 1) & 31] : x;   // lane 31's neighbour
            float2 xn;
            xn.x = __shfl_sync(0xffffffffu, pv.x, (l + 1) & 31);
            xn.y = __shfl_sync(0xffffffffu, pv.y, (l + 1) & 31);
            const float2 d = x - xn;
            const float ph = kHalfBinScale * fmaf(d.x, d.x, d.y * d.y);
            if constexpr (i >= 5 && i <= 26) wstore2<OUT>(prow, 2 * (rb + 32 * i), pf, ph);
            else wstore2_if<OUT>(ok, prow, 2 * (rb + 32 * i), pf, ph);
            // an edge register outside the segment can only cause a needless
            // listing pass, which checks every position itself
            mx = fmaxf(mx, fmaxf(pf, ph));
        } else {
            if constexpr (i >= 5 && i <= 26) wstore1<OUT>(prow, rb + 32 * i, pf);
            else wstore1_if<OUT>(ok, prow, rb + 32 * i, pf);
            mx = fmaxf(mx, pf);
        }
    });
    return mx;
}

// The general epilogue (a segment reaching the end of the series, overlaps
// above 320) and the listing pass of the fused threshold: the lane's
// registers are staged in position order in the warp's exchange buffer, then
// positions M2 + l, M2 + l + 32, ... below pend are walked by a rolled loop,
// each checked against the series end.  SCAN: list the values above A.thr
// instead of storing.  Returns the lane's largest stored power.
template <int OUT, bool IB, bool SCAN>
__device__ __forceinline__ float wepi_staged(const float2* v, float2* xb, int l, int M2, int pend,
                                             int64_t r0, int64_t npos, void* prow,
                                             const ConvArgs& A, int row, int flags) {
#pragma unroll
    for (int i = 0; i < 32; ++i) xb[l + 32 * i] = v[i];
    __syncwarp();
    float mx = 0.f;
#pragma unroll 1
    for (int p = M2 + l; p < pend; p += 32) {
        const int64_t r = r0 + (p - M2);
        if (r >= npos) break;
        const float2 x = xb[p];
        const float pf = fmaf(x.x, x.x, x.y * x.y);
        if constexpr (IB) {
            const float2 d = x - xb[p + 1];
            // the last bin of the series has no r + 1: its half bin is 0
            const float ph = r + 1 < npos ? kHalfBinScale * fmaf(d.x, d.x, d.y * d.y) : 0.f;
            if constexpr (SCAN) {
                if (pf > A.thr) emit(A, row, 2 * r, pf, flags);
                if (ph > A.thr) emit(A, row, 2 * r + 1, ph, flags);
            } else {
                wstore2<OUT>(prow, 2 * r, pf, ph);
                mx = fmaxf(mx, fmaxf(pf, ph));
            }
        } else {
            if constexpr (SCAN) {
                if (pf > A.thr) emit(A, row, r, pf, flags);
            } else {
                wstore1<OUT>(prow, r, pf);
                mx = fmaxf(mx, pf);
            }
        }
    }
    __syncwarp();
    return mx;
}

// Forward FFT of one segment (a warp's, once per quad): positions base + l +
// 32 i of the series (zero outside it; SUB = 2: the spectrum with zeros
// interleaved, npos = 2 nb), transformed by wfft_forward and left in the
// warp's buffer as xb[i*32 + l] = X[l + 32 i].  (Measured: as a called
// function it was 3 % slower than inlined.)
template <int SUB>
__device__ __forceinline__ void wseg_forward(const float2* __restrict__ spec, int64_t nb, int64_t base,
                                          float2* xb, const float4* tw4, int l) {
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int64_t pos = base + l + 32 * i;
        if constexpr (SUB == 1) {
            v[i] = (pos >= 0 && pos < nb) ? __ldg(&spec[pos]) : make_float2(0.f, 0.f);
        } else {
            v[i] = (pos >= 0 && pos < 2 * nb && !(pos & 1)) ? __ldg(&spec[pos >> 1])
                                                             : make_float2(0.f, 0.f);
        }
    }
    wfft_forward(v, xb, tw4, l);
#pragma unroll
    for (int i = 0; i < 32; ++i) xb[i * 32 + l] = v[i];
    __syncwarp();
}

// PREC 0: the 32-point DFT passes in FP32 on the CUDA cores; PREC 1, 2, 3:
// on the tensor cores (tc_dft.cuh), FP16 hi+lo, BF16 hi+lo, BF16 hi+mid+lo.
// The tensor-core forms hold two CTAs per SM (their DFT matrix parts take
// shared memory, and two CTAs' tensor memory fits the SM's 512 columns).
template <bool FUSE, bool BATCH, int OUT, int SUB, bool IB, int PREC = 0>
__global__ void __launch_bounds__(WShape::NW * 32, PREC ? 2 : kWarpCtasPerSm)
    wconv_kernel(const ConvArgs A) {
    constexpr int NW = WShape::NW, NBUF = WShape::NBUF, ROW4 = WShape::ROW4, L = WShape::L;
    extern __shared__ float4 wsm4[];
    float4* hbuf = wsm4;                                   // NBUF rows of ROW4
    float4* tw4 = hbuf + NBUF * ROW4;
    float2* xall = reinterpret_cast<float2*>(tw4 + WShape::TW4);
    __shared__ uint64_t full[NBUF], empty[NBUF];
    __shared__ volatile int abort_flag;
    __shared__ WProducer<BATCH, SUB> prod;
    __shared__ uint64_t tc_ready, tc_done;
    __shared__ uint32_t tc_tmem;

    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    float2* xb = xall + w * WShape::XBUF;
    const int lo = (int)((int64_t)blockIdx.x * A.items / gridDim.x);
    const int hi = (int)((int64_t)(blockIdx.x + 1) * A.items / gridDim.x);
    if (lo >= hi) return;
    const uint32_t limit = A.wait_limit ? A.wait_limit : kWaitLimit;   // copy-issuing thread

    WWalk<BATCH, SUB> cw;
    cw.init(A, lo);

    // issue the copies of rows up to `target` (thread 0 only)
    auto produce = [&](uint32_t target) {
        while (prod.issued <= target && prod.walk.u < hi) {
            const uint32_t k = prod.issued, b = k % NBUF;
            if (k >= NBUF && !wwait(&empty[b], ((k / NBUF) - 1) & 1, &abort_flag, limit)) {
                if (!abort_flag && A.status) atomicOr(A.status, FDAS_STATUS_TIMEOUT);
                abort_flag = 1;
                return;
            }
            int row, brow, cj;
            item_row(A, prod.walk.grp, prod.walk.q, row, brow, cj);
            fence_proxy_async();
            if (A.probe && k == 0) {   // diagnostic: armed, never filled
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             ::"r"(smem_u32(&full[b])), "r"((uint32_t)(ROW4 * sizeof(float4)))
                             : "memory");
            } else {
                tma_load_1d(hbuf + b * ROW4, A.bank + (size_t)brow * ROW4,
                            ROW4 * sizeof(float4), &full[b]);
            }
            prod.issued = k + 1;
            // skip the units that use the same row (a +-z pair, a one-row group)
            int r2, b2 = brow, c2;
            do {
                prod.walk.advance(A);
                if (prod.walk.u >= hi) break;
                item_row(A, prod.walk.grp, prod.walk.q, r2, b2, c2);
            } while (b2 == brow);
        }
    };

    wfft_twiddles(tw4, tid, NW * 32);
    constexpr int TP = PREC ? PREC : 1;
    unsigned char* wparts = reinterpret_cast<unsigned char*>(xall + NW * WShape::XBUF);
    if constexpr (PREC != 0) {
        tc_fill_w<TP>(wparts, tid, NW * 32);
        fence_proxy_async();   // the DFT matrix is read by the tensor cores
        if (w == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         ::"r"(smem_u32(&tc_tmem)), "r"((uint32_t)TcShape<TP>::NCOLS) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], NW);
        }
        if constexpr (PREC != 0) {
            mbar_init(&tc_ready, NW);
            mbar_init(&tc_done, 1);
        }
        abort_flag = 0;
        prod.walk = cw;
        prod.issued = 0;
        produce(NBUF - 1);
    }
    if constexpr (PREC != 0) tc_fence_before();
    __syncthreads();
    TcCtx tc;
    if constexpr (PREC != 0) {
        tc_fence_after();
        tc.tmem = tc_tmem;
        tc.wsm = smem_u32(wparts);
        tc.ready = &tc_ready;
        tc.done = &tc_done;
        tc.phase = 0;
        tc.commits = 0;
    }
    // one 32-point DFT pass of the inverse (PREC 0: in registers)
    auto pass = [&](float2* x) -> bool {
        if constexpr (PREC == 0) {
            dft32<1>(x);
            return true;
        } else {
            return tc_dft32<TP>(x, tc, tid, &abort_flag, limit);
        }
    };
    // the inverse transform, k = l + 32 i -> p = l + 32 i (wfft_inverse's steps)
    auto inverse = [&](float2* x) -> bool {
#pragma unroll 1
        for (int ps = 0; ps < 2; ++ps) {
            if (!pass(x)) return false;
            if (ps == 0) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float4 t = tw4[j * 32 + l];
                    if (j) x[2 * j] = cmul(x[2 * j], make_float2(t.x, t.y));
                    x[2 * j + 1] = cmul(x[2 * j + 1], make_float2(t.z, t.w));
                }
                wfft_transpose(x, xb, l);
            }
        }
        return true;
    };

    float2 Y[32], v[32];
    bool fresh = true, live = false;
    int cur_brow = -1, M2 = 0;
    int r0 = 0, npos = 0;
    uint32_t ri = 0xffffffffu;   // index of the row in use
    while (cw.u < hi) {
        int row, brow, cj;
        item_row(A, cw.grp, cw.q, row, brow, cj);
        if (fresh) {
            // ---- a new quad: this warp's segment, its geometry and forward FFT ----
            M2 = A.gM[cw.grp] / 2;
            const int B = L - 2 * M2;
            npos = (int)cw.npos(A);
            r0 = (cw.quad * NW + w) * B;   // bin of position M/2
            live = r0 < npos;
            if constexpr (PREC == 0) {
                if (live) {
                    wseg_forward<SUB>(cw.ser.spec(A), cw.ser.nb(A), r0 - M2, xb, tw4, l);
#pragma unroll
                    for (int i = 0; i < 32; ++i) Y[i] = xb[i * 32 + l];
                    __syncwarp();
                }
            } else {
                // every warp takes part in the CTA's tensor-core passes (a segment
                // past the series transforms zeros); forward = conj(inverse(conj))
                const float2* sp = cw.ser.spec(A);
                const int64_t base = r0 - M2 + l, nbs = cw.ser.nb(A);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int64_t pos = base + 32 * i;
                    float2 z;
                    if constexpr (SUB == 1) {
                        z = (pos >= 0 && pos < nbs) ? __ldg(&sp[pos]) : make_float2(0.f, 0.f);
                    } else {
                        z = (pos >= 0 && pos < 2 * nbs && !(pos & 1)) ? __ldg(&sp[pos >> 1])
                                                                      : make_float2(0.f, 0.f);
                    }
                    Y[i] = make_float2(z.x, -z.y);
                }
                if (!inverse(Y)) break;
#pragma unroll
                for (int i = 0; i < 32; ++i) Y[i].y = -Y[i].y;
            }
        }
        if (brow != cur_brow) {
            // ---- release the previous row, wait for this one ----
            if (cur_brow >= 0) {
                __syncwarp();
                if (l == 0) mbar_arrive(&empty[ri % NBUF]);
            }
            ++ri;
            cur_brow = brow;
            if (tid == 0) produce(ri + NBUF - 1);
            const bool got = wwait(&full[ri % NBUF], (ri / NBUF) & 1, &abort_flag,
                                   A.wait_limit ? A.wait_limit : kWaitLimit);
            if (!__all_sync(0xffffffffu, got)) {   // the warp leaves together
                if (l == 0) {
                    if (!abort_flag && A.status) atomicOr(A.status, FDAS_STATUS_TIMEOUT);
                    abort_flag = 1;
                }
                break;
            }
        }
        if (live || PREC != 0) {
            // ---- multiply by the template spectrum ----
            const float4* hr = hbuf + (ri % NBUF) * ROW4;
            if (!cj) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float4 h = hr[j * 33 + l];
                    v[2 * j] = cmul_p(Y[2 * j], make_float2(h.x, h.y));
                    v[2 * j + 1] = cmul_p(Y[2 * j + 1], make_float2(h.z, h.w));
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float4 h = hr[527 - 33 * j - l];
                    v[2 * j] = cmulc_p(Y[2 * j], make_float2(h.z, h.w));
                    v[2 * j + 1] = cmulc_p(Y[2 * j + 1], make_float2(h.x, h.y));
                }
            }
            // ---- inverse FFT ----
            if constexpr (PREC == 0) {
                wfft_inverse(v, xb, tw4, l);
            } else {
                if (!inverse(v)) break;
                if (!live) {
                    fresh = cw.advance(A);
                    continue;
                }
            }
            // ---- powers of positions M/2 .. M/2 + B - 1 ----
            void* prow = OUT == 0 ? static_cast<void*>(cw.ser.plane(A) + (int64_t)row * cw.ser.row_stride(A))
                                  : static_cast<void*>(reinterpret_cast<uint16_t*>(cw.ser.plane(A)) +
                                                       (int64_t)row * cw.ser.row_stride(A));
            float mx;
            if (M2 <= 160 && r0 + L - 2 * M2 <= npos) {
                // first registers at positions >= M/2 and >= M/2 + B
                mx = wepi_fast<OUT, IB>(v, l, (M2 - l + 31) >> 5, (L - M2 - l + 31) >> 5, prow,
                                        r0 - M2 + l);
            } else {
                mx = wepi_staged<OUT, IB, false>(v, xb, l, M2, L - M2, r0, npos, prow, A, row, 0);
            }
            if constexpr (FUSE) {
                if (__any_sync(0xffffffffu, mx > A.thr))   // rare: list the crossings
                    wepi_staged<OUT, IB, true>(v, xb, l, M2, L - M2, r0, npos, prow, A, row,
                                               cw.ser.flags());
            }
        }
        fresh = cw.advance(A);
    }

    if (tid == 0 && abort_flag) {
        // no copy may still be writing this CTA's shared memory when it exits
        const uint32_t n = prod.issued;
        for (uint32_t k = (n > NBUF ? n - NBUF : 0); k < n; ++k) {
            if (A.probe && k == 0) continue;   // armed without a copy: nothing in flight
            const int never = 0;
            wwait(&full[k % NBUF], (k / NBUF) & 1, &never, limit);
        }
        if constexpr (PREC != 0) {
            // nor may tensor-core products still be running on its tensor memory
            if (tc.commits > 0) mbar_wait_bounded(&tc_done, (tc.commits - 1) & 1u, limit);
        }
    }
    if constexpr (PREC != 0) {
        // every wait above is bounded, so every thread arrives here
        tc_fence_before();
        __syncthreads();
        if (w == 0) {
            tc_fence_after();
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                         ::"r"(tc.tmem), "r"((uint32_t)TcShape<TP>::NCOLS) : "memory");
        }
    }
}

template <bool FUSE, bool BATCH, int OUT, int SUB, bool IB, int PREC = 0>
static int launch_w(const ConvArgs& args, int ctas_per_sm, cudaStream_t st) {
    constexpr size_t smem = WSmem<PREC>::bytes;
    // unit indices are 32-bit in the kernel (2^31 units of 4 segments would
    // be a plane of more than 8 TB)
    if (args.items > 0x7fffffff) return FDAS_E_UNSUPPORTED;
    int sms = 0, max_per_sm = 0;
    const int rc = kernel_setup(
        reinterpret_cast<const void*>(&wconv_kernel<FUSE, BATCH, OUT, SUB, IB, PREC>), smem,
        WShape::NW * 32, &sms, &max_per_sm);
    if (rc != FDAS_OK) return rc;
    int per = (ctas_per_sm > 0 && ctas_per_sm < max_per_sm) ? ctas_per_sm : max_per_sm;
    // tensor memory: the CTAs resident on an SM must fit its 512 columns, or
    // an allocation would wait for another CTA to finish
    if (PREC != 0) per = std::min(per, 512 / TcShape<PREC ? PREC : 1>::NCOLS);
    if (PREC != 0 && max_per_sm > 512 / TcShape<PREC ? PREC : 1>::NCOLS) return FDAS_E_UNSUPPORTED;
    const int64_t g = std::min<int64_t>((int64_t)sms * per, std::max<int64_t>(1, args.items));
    wconv_kernel<FUSE, BATCH, OUT, SUB, IB, PREC><<<(unsigned)g, WShape::NW * 32, smem, st>>>(args);
    return cuda_status(cudaGetLastError());
}

}  // namespace fdas
