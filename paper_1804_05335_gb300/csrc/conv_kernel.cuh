// The fused overlap-save convolver kernel (Sections 3, 4.1, 4.2), shared by
// the translation units that instantiate its FP32 and split-precision forms.
//
// One persistent CTA per SM slot walks a contiguous, statically balanced
// range of (segment, template) work items in segment-major order.  For each
// new segment it loads the L spectrum bins starting at s*B - M/2 (zero
// outside [0, nb)) and runs the forward FFT once; for every template it
// multiplies by the template spectrum, runs the inverse FFT, forms full- and
// half-bin powers of the B useful outputs and writes them to the plane with
// 16-byte coalesced stores.  Nothing but the plane (and optional candidates)
// is written to global memory.
//
// FFT layout (L = 16*16*Q, T = L/16 threads, 16 complex values per thread):
// the forward transform is decimation-in-frequency in three register passes
// (radix 16, 16, Q) separated by shared-memory exchanges, and leaves the
// spectrum digit-reversed; the inverse is the transposed decimation-in-time
// sequence (radix Q, 16, 16), which takes digit-reversed input and returns
// natural order.  The pointwise product therefore never needs the reordering
// permutation (Section 4.2), and the template bank is stored in the same
// digit-reversed order.  Thread/register distributions (p = position):
//   D1: thread t, reg i          p = i*T + t
//   D2: thread t = a*Q + c, reg b  p = a*T + b*Q + c
//   D3: thread t = a*Q + c, reg i = s*Q + c2   p = a*T + (c + Q*s)*Q + c2
// D2 <-> D3 exchanges stay inside a group of Q threads (one warp), D1 <-> D2
// needs the whole CTA.  Both shared-memory layouts are padded so that every
// exchange is free of bank conflicts.
//
// z < 0 templates of a symmetric grid use H_{-z}[k] = conj(H_z[-k mod L])
// (Section 4.2): in D3, -k of (thread t, reg i) lives in (partner(t), 15-i)
// except for thread 0, handled separately.
//
// SUB = 2 samples the correlation at every half bin (2-bin Fourier
// interpolation): the segments are cut from the spectrum with zeros
// interleaved, 2 nb positions, and the bank holds half-bin templates.
// OUT selects the plane element type (0 float, 1 binary16, 2 bfloat16).
// PREC selects the arithmetic of the four radix-16 passes: 0 = FP32 on the
// CUDA cores; 1, 2 = split-precision tensor-core products (split_mma.cuh,
// FP16 or BF16 hi+lo operands, FP32 accumulation).  The radix-Q passes, the
// twiddles, the template product and the power stay FP32 in every form.
#pragma once
#include "conv_common.cuh"
#include "conv_fft.cuh"
#include "split_mma.cuh"
#include "tma.cuh"

namespace fdas {

template <int L>
struct ConvSmem {
    using S = ConvShape<L>;
    static constexpr int TW3 = 16 * (S::Q + 1);
    // buf0 | buf1 | outb (L) | hbuf (bank row) | tw3
    static constexpr size_t bytes = (size_t)(2 * S::BUFS + L + S::ROW + TW3) * sizeof(float2);
};

template <int L, bool FUSE, bool BATCH, int PREC, int OUT, int SUB>
__global__ void __launch_bounds__(L / 16, L == 2048 ? 2 : 1) conv_kernel(const ConvArgs A) {
    using S = ConvShape<L>;
    constexpr int T = S::T, Q = S::Q, G = S::G, BUFS = S::BUFS, NS = S::NS;
    extern __shared__ float4 smem4[];
    float2* buf0 = reinterpret_cast<float2*>(smem4);
    float2* buf1 = buf0 + BUFS;
    float2* outb = buf1 + BUFS;
    float2* hbuf = outb + L;
    float2* tw3 = hbuf + S::ROW;
    __shared__ uint64_t hbar;

    const int t = threadIdx.x;
    const int a = t / Q, c = t % Q;
    int M = A.M, B = L - M, NP = B / 2;   // of the current item's group

    const int64_t lo = (int64_t)blockIdx.x * A.items / gridDim.x;
    const int64_t hi = (int64_t)(blockIdx.x + 1) * A.items / gridDim.x;
    if (lo >= hi) return;
    int trial = 0;
    if constexpr (BATCH) {
        // last trial whose first item is <= lo
        int a0 = 0, a1 = A.ntrials - 1;
        while (a0 < a1) {
            const int mid = (a0 + a1 + 1) >> 1;
            if (A.trials[mid].item_begin <= lo) a0 = mid; else a1 = mid - 1;
        }
        trial = a0;
    }
    SeriesState st = series_of<BATCH>(A, trial);
    // correlation positions of the series: its bins, or twice as many with
    // half-bin sampling (SUB = 2: the spectrum with zeros interleaved)
    auto npos = [&]() -> int64_t { return SUB * st.nb; };
    const int64_t first = BATCH ? A.trials[trial].item_begin : 0;
    // group, segment and template of the first item
    int grp = 0;
    int64_t rel = lo - first;
    int64_t gseg = group_segments(A, L, 0, npos());
    while (rel >= gseg * A.gK[grp] && grp + 1 < A.ng) {
        rel -= gseg * A.gK[grp];
        ++grp;
        gseg = group_segments(A, L, grp, npos());
    }
    M = A.gM[grp];
    B = L - M;
    NP = B / 2;
    int64_t s = rel / A.gK[grp];
    int q = (int)(rel - s * A.gK[grp]);
    int row, brow, cj;
    item_row(A, grp, q, row, brow, cj);

    if (t == 0) {
        mbar_init(&hbar, 1);
        tma_load_1d(hbuf, A.bank + (size_t)brow * (S::ROW / 2), S::ROW * sizeof(float2), &hbar);
    }
    // inverse pass-3' twiddles: tw3[k1*(Q+1) + n2] = exp(+i 2 pi n2 k1 / (L/16))
    for (int idx = t; idx < ConvSmem<L>::TW3; idx += T) {
        int k1 = idx / (Q + 1), n2 = idx % (Q + 1);
        float sn, cs;
        sincospif(2.0f * (float)((n2 * k1) % (L / 16)) / (float)(L / 16), &sn, &cs);
        tw3[idx] = make_float2(cs, sn);
    }
    // inverse pass-2' twiddles (thread (a, c), reg n1): exp(+i 2 pi (n1 Q + c) a / L)
    // Split forms hold, per lane, the twiddles of its four MMA instances
    // (split_mma.cuh): tw2[4*mi + j] for instance mi, output n1 = tig + 4 j.
    float2 tw2[16];
    const MmaLane ml(t);
    if constexpr (PREC == 0) {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            float sn, cs;
            sincospif(2.0f * (float)(((n1 * Q + c) * a) % L) / (float)L, &sn, &cs);
            tw2[n1] = make_float2(cs, sn);
        }
    } else {
#pragma unroll
        for (int mi = 0; mi < 4; ++mi)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int tm = ml.inst(mi), am = tm / Q, cm = tm % Q;
                float sn, cs;
                sincospif(2.0f * (float)((((ml.tig + 4 * j) * Q + cm) * am) % L) / (float)L, &sn, &cs);
                tw2[4 * mi + j] = make_float2(cs, sn);
            }
    }
    SplitMMA<PREC == 0 ? 1 : PREC> iw;   // inverse DFT matrix (unused by PREC 0)
    if constexpr (PREC != 0) iw.template init<1>(ml.lane);
    // conjugate (z < 0) templates read H[-k]: float4 pair ip of this thread
    // sits at hbase - ip*hstep, halves swapped (partner thread, reversed
    // registers); thread 0 reads the mirror slots at the end of the row.
    const int tp = (a != 0) ? (16 - a) * Q + (Q - 1 - c) : (Q - c) % Q;
    const int hbase = (t == 0) ? L / 2 + 7 : 7 * T + tp;
    const int hstep = (t == 0) ? 1 : T;
    __syncthreads();

    int64_t cur_seg = -1;   // segment (and group) of the forward FFT held in Y
    int cur_grp = -1;
    int parity = 0;
    uint32_t hphase = 0;
    bool hpending = true;
    float2 Y[16];
    float2 v[16];
    const float4* hb4 = reinterpret_cast<const float4*>(hbuf);

    for (int64_t w = lo; w < hi; ++w) {
        if constexpr (BATCH) {
            if (w == st.end) {   // next trial: its first segment and template
                ++trial;
                st = series_of<BATCH>(A, trial);
                s = 0;
                q = 0;
                grp = 0;
                gseg = group_segments(A, L, 0, npos());
                M = A.gM[0];
                B = L - M;
                NP = B / 2;
                item_row(A, 0, 0, row, brow, cj);
                cur_seg = -1;
            }
        }
        if (s != cur_seg || grp != cur_grp) {
            // ---- forward FFT of segment s, once per segment (and group) ----
            cur_seg = s;
            cur_grp = grp;
            const int64_t base = s * (int64_t)B - M / 2;
            if constexpr (PREC == 0) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int64_t pos = base + i * T + t;
                    if constexpr (SUB == 1) {
                        v[i] = (pos >= 0 && pos < st.nb) ? __ldg(&st.spec[pos]) : make_float2(0.f, 0.f);
                    } else {   // the spectrum with zeros interleaved (2-bin interpolation)
                        v[i] = (pos >= 0 && pos < npos() && !(pos & 1)) ? __ldg(&st.spec[pos >> 1])
                                                                          : make_float2(0.f, 0.f);
                    }
                }
                forward_fft_d3<L>(v, buf0, buf1, t);
            } else {
                forward_fft_d3_split<L, PREC>(st.spec, st.nb, base, v, buf0, buf1, t);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) Y[i] = v[i];
            __syncthreads();   // exchange buffers free again
            parity = 0;
        }

        // ---- multiply by the template spectrum staged in shared memory ----
        bool tmo = false;
        if (hpending) {
            tmo = !mbar_wait_bounded(&hbar, hphase, kWaitLimit);
            hphase ^= 1u;
            hpending = false;
        }
        if (!cj) {
#pragma unroll
            for (int ip = 0; ip < 8; ++ip) {
                const float4 h = hb4[ip * T + t];
                v[2 * ip] = cmul(Y[2 * ip], make_float2(h.x, h.y));
                v[2 * ip + 1] = cmul(Y[2 * ip + 1], make_float2(h.z, h.w));
            }
        } else {
#pragma unroll
            for (int ip = 0; ip < 8; ++ip) {
                const float4 h = hb4[hbase - ip * hstep];
                v[2 * ip] = cmulc(Y[2 * ip], make_float2(h.z, h.w));
                v[2 * ip + 1] = cmulc(Y[2 * ip + 1], make_float2(h.x, h.y));
            }
        }

        // ---- inverse pass 3': radix Q over k2, then twiddle ----
#pragma unroll
        for (int s2 = 0; s2 < NS; ++s2) {
            dftq<Q, 1>(v + s2 * Q);
#pragma unroll
            for (int n2 = 1; n2 < Q; ++n2)
                v[s2 * Q + n2] = cmul(v[s2 * Q + n2], tw3[(c + Q * s2) * (Q + 1) + n2]);
        }
        // ---- D3 -> D2 inside the Q-thread group ----
        float2* x1 = parity ? buf1 : buf0;
        {
            float2* x2b = parity ? buf0 : buf1;
            float2* x2 = x2b + a * G;
#pragma unroll
            for (int i = 0; i < 16; ++i) x2[(c + Q * (i / Q)) * (Q + 1) + (i % Q)] = v[i];
            __syncwarp();
            if constexpr (PREC == 0) {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = x2[i * (Q + 1) + c];
                // ---- inverse pass 2': radix 16 over k1, then twiddle ----
                dft16<1>(v);
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1) v[n1] = cmul(v[n1], tw2[n1]);
                // ---- D2 -> D1 across the CTA ----
#pragma unroll
                for (int i = 0; i < 16; ++i) x1[a * (T + Q) + i * Q + c] = v[i];
            } else {
                // the same pass over the warp's 32 instances on tensor cores
                float2 xm[4][4], ym[4][4];
#pragma unroll
                for (int mi = 0; mi < 4; ++mi) {
                    const int tm = ml.inst(mi);
                    const float2* xb = x2b + (tm / Q) * G + tm % Q;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) xm[mi][kk] = xb[(ml.tig + 4 * kk) * (Q + 1)];
                }
                iw.apply(xm, ym);
#pragma unroll
                for (int mi = 0; mi < 4; ++mi) {
                    const int tm = ml.inst(mi);
                    float2* xo = x1 + (tm / Q) * (T + Q) + tm % Q;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        xo[(ml.tig + 4 * j) * Q] = cmul(ym[mi][j], tw2[4 * mi + j]);
                }
            }
        }
        if (__syncthreads_or(tmo)) {
            if (t == 0) {
                if (A.status) atomicOr(A.status, FDAS_STATUS_TIMEOUT);
                // the row's copy may still be in flight: wait for it (bounded)
                // before the CTA's shared memory is released
                mbar_wait_bounded(&hbar, hphase ^ 1u, kWaitLimit);
            }
            break;
        }

        // ---- next item; prefetch its template row if it changes ----
        int64_t s_next = s;
        int q_next = q + 1, grp_next = grp;
        if (q_next == A.gK[grp]) {
            q_next = 0;
            if (++s_next == gseg) {
                s_next = 0;
                // the series is done after its last group; a batched launch
                // continues with the next series' first group
                if (++grp_next == A.ng) grp_next = 0;
            }
        }
        int row_n = 0, brow_n = brow, cj_n = 0;
        if (w + 1 < hi) {
            item_row(A, grp_next, q_next, row_n, brow_n, cj_n);
            if (brow_n != brow) {
                if (t == 0) {
                    fence_proxy_async();
                    tma_load_1d(hbuf, A.bank + (size_t)brow_n * (S::ROW / 2), S::ROW * sizeof(float2),
                                &hbar);
                }
                hpending = true;
            }
        }

        if constexpr (PREC == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = x1[i * (T + Q) + t];
            // ---- inverse pass 1': radix 16 over k0 -> natural order ----
            dft16<1>(v);
#pragma unroll
            for (int n0 = 0; n0 < 16; ++n0) outb[n0 * T + t] = v[n0];
        } else {
            float2 xm[4][4], ym[4][4];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    xm[mi][kk] = x1[(ml.tig + 4 * kk) * (T + Q) + ml.inst(mi)];
            iw.apply(xm, ym);
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int j = 0; j < 4; ++j) outb[(ml.tig + 4 * j) * T + ml.inst(mi)] = ym[mi][j];
        }
        __syncthreads();

        // ---- epilogue: powers of positions M/2 .. M/2+B, two bins per pair ----
        const int64_t r0 = s * (int64_t)B;
        // plane row (elements of type OUT)
        void* prow = OUT == 0 ? static_cast<void*>(st.plane + (int64_t)row * st.row_stride)
                              : static_cast<void*>(reinterpret_cast<uint16_t*>(st.plane) +
                                                   (int64_t)row * st.row_stride);
        const float4* o4 = reinterpret_cast<const float4*>(outb + M / 2);
        const float2* o2 = outb + M / 2 + 2;
        float mx = 0.f;
        if (r0 + B < npos()) {
            constexpr int UMAX = (L / 2 - 32 + T - 1) / T;   // pairs per thread for M >= 64
            auto pair_ib = [&](int p) {
                const float4 pw = pair_powers(o4[p], o2[2 * p]);
                plane_store4<OUT>(prow, 2 * r0 + 4 * p, pw);
                if constexpr (FUSE) mx = fmaxf(mx, fmaxf(fmaxf(pw.x, pw.y), fmaxf(pw.z, pw.w)));
            };
            auto pair_full = [&](int p) {
                const float4 x = o4[p];
                const float2 pw = make_float2(fmaf(x.x, x.x, x.y * x.y), fmaf(x.z, x.z, x.w * x.w));
                plane_store2<OUT>(prow, r0 + 2 * p, pw);
                if constexpr (FUSE) mx = fmaxf(mx, fmaxf(pw.x, pw.y));
            };
            // with NP >= (UMAX - 1) T (overlaps up to L - 2 (UMAX - 1) T) only a
            // thread's last pair can fall past NP
            const bool head = NP >= (UMAX - 1) * T;
            if (A.interbin == 1) {
                if (head) {
#pragma unroll
                    for (int u = 0; u < UMAX - 1; ++u) pair_ib(t + u * T);
                    if (t + (UMAX - 1) * T < NP) pair_ib(t + (UMAX - 1) * T);
                } else {
#pragma unroll
                    for (int u = 0; u < UMAX; ++u)
                        if (t + u * T < NP) pair_ib(t + u * T);
                }
            } else {
                if (head) {
#pragma unroll
                    for (int u = 0; u < UMAX - 1; ++u) pair_full(t + u * T);
                    if (t + (UMAX - 1) * T < NP) pair_full(t + (UMAX - 1) * T);
                } else {
#pragma unroll
                    for (int u = 0; u < UMAX; ++u)
                        if (t + u * T < NP) pair_full(t + u * T);
                }
            }
        } else {
            // segment reaching the end of the spectrum: per-bin checks
            for (int p = t; p < NP; p += T) {
                const int64_t r = r0 + 2 * p;
                if (r >= npos()) break;
                float4 pw = pair_powers(o4[p], o2[2 * p]);
                if (r + 1 >= npos() - 1) pw.w = 0.f;       // no bin r+2
                if (r >= npos() - 1) pw.y = 0.f;           // no bin r+1
                if (r + 1 >= npos()) { pw.z = 0.f; pw.w = 0.f; }
                if (A.interbin == 1) {
                    plane_store1<OUT>(prow, 2 * r, pw.x);
                    plane_store1<OUT>(prow, 2 * r + 1, pw.y);
                    if (r + 1 < npos()) {
                        plane_store1<OUT>(prow, 2 * r + 2, pw.z);
                        plane_store1<OUT>(prow, 2 * r + 3, pw.w);
                    }
                } else {
                    plane_store1<OUT>(prow, r, pw.x);
                    if (r + 1 < npos()) plane_store1<OUT>(prow, r + 1, pw.z);
                    pw.y = 0.f;
                    pw.w = 0.f;
                }
                if constexpr (FUSE) mx = fmaxf(mx, fmaxf(fmaxf(pw.x, pw.y), fmaxf(pw.z, pw.w)));
            }
        }
        if constexpr (FUSE) {
            if (mx > A.thr) {
                // rare: rescan this thread's pairs and emit each crossing
                for (int p = t; p < NP; p += T) {
                    const int64_t r = r0 + 2 * p;
                    if (r >= npos()) break;
                    float4 pw = pair_powers(o4[p], o2[2 * p]);
                    if (r + 1 >= npos() - 1) pw.w = 0.f;
                    if (r >= npos() - 1) pw.y = 0.f;
                    if (r + 1 >= npos()) { pw.z = 0.f; pw.w = 0.f; }
                    if (A.interbin == 1) {
                        if (pw.x > A.thr) emit(A, row, 2 * r, pw.x, st.flags);
                        if (pw.y > A.thr) emit(A, row, 2 * r + 1, pw.y, st.flags);
                        if (pw.z > A.thr) emit(A, row, 2 * r + 2, pw.z, st.flags);
                        if (pw.w > A.thr) emit(A, row, 2 * r + 3, pw.w, st.flags);
                    } else {
                        if (pw.x > A.thr) emit(A, row, r, pw.x, st.flags);
                        if (pw.z > A.thr) emit(A, row, r + 1, pw.z, st.flags);
                    }
                }
            }
        }
        parity ^= 1;
        s = s_next;
        q = q_next;
        if (grp_next != grp) {
            grp = grp_next;
            gseg = group_segments(A, L, grp, npos());
            M = A.gM[grp];
            B = L - M;
            NP = B / 2;
        }
        row = row_n;
        brow = brow_n;
        cj = cj_n;
    }
}

template <int L, bool FUSE, bool BATCH, int PREC = 0, int OUT = 0, int SUB = 1>
static int launch_one(const ConvArgs& args, int ctas_per_sm, cudaStream_t st) {
    using S = ConvShape<L>;
    constexpr size_t smem = ConvSmem<L>::bytes;
    int sms = 0, max_per_sm = 0;
    const int rc = kernel_setup(reinterpret_cast<const void*>(
                                    &conv_kernel<L, FUSE, BATCH, PREC, OUT, SUB>),
                                smem, S::T, &sms, &max_per_sm);
    if (rc != FDAS_OK) return rc;
    const int per = (ctas_per_sm > 0 && ctas_per_sm < max_per_sm) ? ctas_per_sm : max_per_sm;
    const int64_t g = std::min<int64_t>((int64_t)sms * per, std::max<int64_t>(1, args.items));
    conv_kernel<L, FUSE, BATCH, PREC, OUT, SUB><<<(unsigned)g, S::T, smem, st>>>(args);
    return cuda_status(cudaGetLastError());
}

}  // namespace fdas
