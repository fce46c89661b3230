// Argument validation, grid bookkeeping and the small C-ABI helpers.
#include <stdlib.h>

#include <map>
#include <mutex>
#include <utility>

#include "internal.h"

namespace fdas {

static int32_t half_width_i(int32_t z) {
    int32_t az = z < 0 ? -z : z;
    return (az + 1) / 2 + 8;   // ceil(|z|/2) + 8
}

// Splits a symmetric grid's bank rows (z >= 0, |z| increasing) into at most
// kMaxGroups runs of consecutive rows.  A template of half-width h needs an
// overlap of at least 2h + 2 points (h on each side plus the half bin's
// neighbour), rounded up to a multiple of 4 and at least 64; a group uses the
// overlap of its last (widest) row.  The split minimises the convolver's
// work, sum over groups of (rows + kSegmentFft) / (L - overlap): a group's
// segments each cost one forward FFT plus one pass per template, and the
// forward FFT (no template product, no powers) costs about half a pass.  Dynamic programming over the runs of rows that
// need the same overlap.
// The overlap only moves the segment boundaries: the correlation values are
// the same for every overlap that fits the template.  Other grids: one group
// with overlap M.
constexpr double kSegmentFft = 0.5;

static void plan_groups(const fdas_params* p, Grid* g) {
    g->ng = 1;
    g->gM[0] = p->M;
    g->gb0[0] = 0;
    g->gK[0] = g->K;
    if (!g->sym) return;
    // runs of equal overlap: run r = bank rows [rs[r], rs[r+1]) with overlap rm[r]
    // (overlaps are multiples of 4 in [64, L/2]: at most 497 runs)
    constexpr int kRuns = 512;
    int rs[kRuns + 1], rm[kRuns], nr = 0;
    for (int b = 0; b < g->Kb; ++b) {
        const int z = p->zmin + (g->j0 + b) * p->zstep;
        int m = ((2 * half_width_i(z) + 2 + 3) / 4) * 4;
        if (m < 64) m = 64;
        if (nr > 0 && rm[nr - 1] == m) continue;
        if (nr == kRuns) return;   // cannot happen for overlaps <= L/2; keep one group
        rs[nr] = b;
        rm[nr] = m;
        ++nr;
    }
    rs[nr] = g->Kb;
    auto rows = [&](int r0, int r1) {
        return 2 * (rs[r1] - rs[r0]) - ((g->zero && rs[r0] == 0) ? 1 : 0);
    };
    // best[k][r]: runs [0, r) in k groups
    double best[kMaxGroups + 1][kRuns + 1];
    int from[kMaxGroups + 1][kRuns + 1];
    for (int k = 0; k <= kMaxGroups; ++k)
        for (int r = 0; r <= nr; ++r) best[k][r] = 1e300;
    best[0][0] = 0.0;
    for (int k = 1; k <= kMaxGroups; ++k)
        for (int r1 = 1; r1 <= nr; ++r1)
            for (int r0 = 0; r0 < r1; ++r0) {
                if (best[k - 1][r0] >= 1e300) continue;
                const double c = best[k - 1][r0] +
                                 ((double)rows(r0, r1) + kSegmentFft) / (double)(p->L - rm[r1 - 1]);
                if (c < best[k][r1]) {
                    best[k][r1] = c;
                    from[k][r1] = r0;
                }
            }
    int kb = 1;
    for (int k = 2; k <= kMaxGroups; ++k)
        if (best[k][nr] < best[kb][nr] * (1.0 - 1e-9)) kb = k;
    int ends[kMaxGroups + 1];
    for (int k = kb, r = nr; k >= 0; --k) {
        ends[k] = r;
        if (k > 0) r = from[k][r];
    }
    g->ng = kb;
    for (int k = 0; k < kb; ++k) {
        g->gb0[k] = rs[ends[k]];
        g->gK[k] = rows(ends[k], ends[k + 1]);
        g->gM[k] = rm[ends[k + 1] - 1];
    }
}

int kernel_setup(const void* fn, size_t smem, int threads, int* sms, int* per_sm, int carveout) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, std::pair<int, int>> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FDAS_E_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find({fn, dev});
    if (it == done.end()) {
        int n = 0, per = 0;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            (carveout >= 0 &&
             cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carveout) !=
                 cudaSuccess) ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess)
            return FDAS_E_CUDA;
        it = done.emplace(std::make_pair(fn, dev), std::make_pair(n, per)).first;
    }
    if (sms) *sms = it->second.first;
    if (per_sm) *per_sm = it->second.second;
    return it->second.second >= 1 ? FDAS_OK : FDAS_E_UNSUPPORTED;
}

int make_grid(const fdas_params* p, Grid* g) {
    if (!p || !g) return FDAS_E_INVAL;
    if (p->L != 1024 && p->L != 2048 && p->L != 4096) return FDAS_E_INVAL;
    if (p->M < 64 || p->M > p->L / 2 || (p->M % 4) != 0) return FDAS_E_INVAL;
    if (p->zstep < 1 || p->zmin > p->zmax) return FDAS_E_INVAL;
    if ((int64_t)p->zmax - (int64_t)p->zmin > 100000) return FDAS_E_INVAL;
    if ((p->zmax - p->zmin) % p->zstep != 0) return FDAS_E_INVAL;
    if (p->interbin < 0 || p->interbin > 2) return FDAS_E_INVAL;
    int32_t zabs = abs(p->zmin) > abs(p->zmax) ? abs(p->zmin) : abs(p->zmax);
    int32_t hmax = half_width_i(zabs);
    // the template must fit the discarded edge: h taps each side (2h at half-bin
    // sampling), plus the neighbour of the half bin
    if (p->interbin == 2 ? 4 * hmax + 2 > p->M : hmax > p->M / 2 - 1) return FDAS_E_INVAL;
    g->K = (p->zmax - p->zmin) / p->zstep + 1;
    g->hmax = hmax;
    // +-z conjugate pairing needs integer tap offsets: not with half-bin sampling
    g->sym = (p->zmin == -p->zmax && p->zmax > 0 && p->interbin != 2) ? 1 : 0;
    if (g->sym) {
        int32_t j0 = 0;
        while (j0 < g->K && p->zmin + j0 * p->zstep < 0) ++j0;
        g->j0 = j0;
        g->Kb = g->K - j0;
        g->zero = (p->zmin + j0 * p->zstep == 0) ? 1 : 0;
    } else {
        g->j0 = 0;
        g->Kb = g->K;
        g->zero = 0;
    }
    plan_groups(p, g);
    return FDAS_OK;
}

int64_t series_items(const Grid& g, int L, int64_t npos) {
    int64_t items = 0;
    for (int k = 0; k < g.ng; ++k) {
        const int64_t B = L - g.gM[k];
        const int64_t segs = (npos + B - 1) / B;
        items += (L == 1024 ? (segs + kWarpSegments - 1) / kWarpSegments : segs) * g.gK[k];
    }
    return items;
}

}  // namespace fdas

using namespace fdas;

extern "C" {

const char* fdas_strerror(int code) {
    switch (code) {
        case FDAS_OK: return "ok";
        case FDAS_E_INVAL: return "invalid argument";
        case FDAS_E_CUDA: return "CUDA error";
        case FDAS_E_OVERFLOW: return "candidate buffer overflow";
        case FDAS_E_TIMEOUT: return "device wait timed out";
        case FDAS_E_UNSUPPORTED: return "unsupported size or device";
        default: return "unknown error";
    }
}

const char* fdas_version(void) { return "0.1.0"; }

int32_t fdas_half_width(int32_t z) { return half_width_i(z); }

int32_t fdas_num_templates(const fdas_params* p) {
    Grid g;
    int rc = make_grid(p, &g);
    return rc == FDAS_OK ? g.K : rc;
}

int32_t fdas_bank_rows(const fdas_params* p) {
    Grid g;
    int rc = make_grid(p, &g);
    return rc == FDAS_OK ? g.Kb : rc;
}

int64_t fdas_bank_floats(const fdas_params* p) {
    Grid g;
    int rc = make_grid(p, &g);
    return rc == FDAS_OK ? (int64_t)g.Kb * bank_row_complex(p->L) * 2 : rc;
}

int64_t fdas_num_segments(const fdas_params* p, int64_t nb) {
    Grid g;
    if (make_grid(p, &g) != FDAS_OK || nb < 1) return FDAS_E_INVAL;
    int64_t B = p->L - p->M;
    return (positions(p, nb) + B - 1) / B;
}

int32_t fdas_template_groups(const fdas_params* p, int32_t* overlap, int32_t* first_row,
                             int32_t* count) {
    Grid g;
    int rc = make_grid(p, &g);
    if (rc != FDAS_OK) return rc;
    for (int k = 0; k < g.ng; ++k) {
        if (overlap) overlap[k] = g.gM[k];
        if (first_row) first_row[k] = g.gb0[k];
        if (count) count[k] = g.gK[k];
    }
    return g.ng;
}

int64_t fdas_plane_width(const fdas_params* p, int64_t nb) {
    Grid g;
    if (make_grid(p, &g) != FDAS_OK || nb < 1) return FDAS_E_INVAL;
    return p->interbin ? 2 * nb : nb;
}

int fdas_make_templates(const fdas_params* p, float* bank, void* stream) {
    Grid g;
    int rc = make_grid(p, &g);
    if (rc != FDAS_OK) return rc;
    if (!bank || !aligned(bank, 16)) return FDAS_E_INVAL;
    return launch_templates(p, g, reinterpret_cast<float2*>(bank), (cudaStream_t)stream);
}

// Argument checks shared by fdas_correlate and fdas_correlate_split.
static int check_correlate(const fdas_params* p, Grid* g, const float* spec, int64_t nb,
                           const float* bank, const float* plane, int64_t row_stride,
                           const fdas_fused_threshold* fused, const int32_t* status) {
    int rc = make_grid(p, g);
    if (rc != FDAS_OK) return rc;
    if (!spec || !bank || !plane || nb < 1 || nb > ((int64_t)1 << 31)) return FDAS_E_INVAL;
    if (!aligned(spec, 8) || !aligned(bank, 16) || !aligned(plane, 16)) return FDAS_E_INVAL;
    int64_t width = p->interbin ? 2 * nb : nb;
    if (row_stride < width || (row_stride % 4) != 0) return FDAS_E_INVAL;
    if (fused) {
        if (!fused->out || !fused->count || fused->cap < 0) return FDAS_E_INVAL;
        if (!aligned(fused->out, 4) || !aligned(fused->count, 4)) return FDAS_E_INVAL;
    }
    if (status && !aligned(status, 4)) return FDAS_E_INVAL;
    return FDAS_OK;
}

int fdas_correlate(const fdas_params* p, const float* spec, int64_t nb, const float* bank,
                   float* plane, int64_t row_stride, const fdas_fused_threshold* fused,
                   int32_t* status, void* stream) {
    Grid g;
    int rc = check_correlate(p, &g, spec, nb, bank, plane, row_stride, fused, status);
    if (rc != FDAS_OK) return rc;
    return launch_correlate(p, g, reinterpret_cast<const float2*>(spec), nb,
                            reinterpret_cast<const float4*>(bank), plane, row_stride, fused,
                            status, (cudaStream_t)stream);
}

int fdas_debug_wait_timeout(const fdas_params* p, const float* spec, int64_t nb, const float* bank,
                            float* plane, int64_t row_stride, uint32_t polls, int32_t* status,
                            void* stream) {
    Grid g;
    int rc = check_correlate(p, &g, spec, nb, bank, plane, row_stride, nullptr, status);
    if (rc != FDAS_OK) return rc;
    if (!status || polls < 1 || polls > (1u << 24)) return FDAS_E_INVAL;
    if (p->L != 1024 || p->interbin == 2) return FDAS_E_UNSUPPORTED;
    return launch_wconv_wait_probe(p, g, reinterpret_cast<const float2*>(spec), nb,
                                   reinterpret_cast<const float4*>(bank), plane, row_stride, polls,
                                   status, (cudaStream_t)stream);
}

int fdas_correlate_plane16(const fdas_params* p, int32_t type, const float* spec, int64_t nb,
                           const float* bank, void* plane, int64_t row_stride,
                           const fdas_fused_threshold* fused, int32_t* status, void* stream) {
    if (type != FDAS_PLANE_F16 && type != FDAS_PLANE_BF16) return FDAS_E_INVAL;
    Grid g;
    int rc = check_correlate(p, &g, spec, nb, bank, static_cast<const float*>(plane), row_stride,
                             fused, status);
    if (rc != FDAS_OK) return rc;
    if (p->interbin == 2) return FDAS_E_UNSUPPORTED;
    return launch_correlate_plane16(p, g, type, reinterpret_cast<const float2*>(spec), nb,
                                    reinterpret_cast<const float4*>(bank), plane, row_stride,
                                    fused, status, (cudaStream_t)stream);
}

int fdas_correlate_split(const fdas_params* p, int32_t prec, const float* spec, int64_t nb,
                         const float* bank, float* plane, int64_t row_stride,
                         const fdas_fused_threshold* fused, int32_t* status, void* stream) {
    if (prec != FDAS_PREC_FP32 && prec != FDAS_PREC_FP16_SPLIT && prec != FDAS_PREC_BF16_SPLIT &&
        prec != FDAS_PREC_BF16_SPLIT3)
        return FDAS_E_INVAL;
    Grid g;
    int rc = check_correlate(p, &g, spec, nb, bank, plane, row_stride, fused, status);
    if (rc != FDAS_OK) return rc;
    if (prec != FDAS_PREC_FP32 && p->interbin == 2) return FDAS_E_UNSUPPORTED;
    if (prec == FDAS_PREC_FP32)
        return launch_correlate(p, g, reinterpret_cast<const float2*>(spec), nb,
                                reinterpret_cast<const float4*>(bank), plane, row_stride, fused,
                                status, (cudaStream_t)stream);
    return launch_correlate_split(p, g, prec, reinterpret_cast<const float2*>(spec), nb,
                                  reinterpret_cast<const float4*>(bank), plane, row_stride, fused,
                                  status, (cudaStream_t)stream);
}

int64_t fdas_batch_plan(const fdas_params* p, fdas_trial* trials, int32_t ntrials) {
    Grid g;
    int rc = make_grid(p, &g);
    if (rc != FDAS_OK) return rc;
    if (!trials || ntrials < 1) return FDAS_E_INVAL;
    int64_t items = 0;
    for (int32_t i = 0; i < ntrials; ++i) {
        fdas_trial& t = trials[i];
        if (!t.spec || !t.plane || t.nb < 1 || t.nb > ((int64_t)1 << 31)) return FDAS_E_INVAL;
        if (!aligned(t.spec, 8) || !aligned(t.plane, 16)) return FDAS_E_INVAL;
        const int64_t width = p->interbin ? 2 * t.nb : t.nb;
        if (t.row_stride < width || (t.row_stride % 4) != 0) return FDAS_E_INVAL;
        t.item_begin = items;
        items += series_items(g, p->L, positions(p, t.nb));
    }
    return items;
}

int fdas_correlate_batched(const fdas_params* p, const fdas_trial* trials, int32_t ntrials,
                           int64_t total_items, const float* bank,
                           const fdas_fused_threshold* fused, const fdas_tuning* tuning,
                           int32_t* status, void* stream) {
    Grid g;
    int rc = make_grid(p, &g);
    if (rc != FDAS_OK) return rc;
    if (!trials || ntrials < 1 || ntrials > (1 << 23) || total_items < 1 || !bank) return FDAS_E_INVAL;
    if (!aligned(trials, 8) || !aligned(bank, 16)) return FDAS_E_INVAL;
    if (fused) {
        if (!fused->out || !fused->count || fused->cap < 0) return FDAS_E_INVAL;
        if (!aligned(fused->out, 4) || !aligned(fused->count, 4)) return FDAS_E_INVAL;
    }
    if (status && !aligned(status, 4)) return FDAS_E_INVAL;
    const int cps = tuning ? tuning->ctas_per_sm : 0;
    const int tpb = tuning ? tuning->templates_per_block : 0;
    if (cps < 0 || tpb < 0) return FDAS_E_INVAL;
    return launch_correlate_batched(p, g, trials, ntrials, total_items,
                                    reinterpret_cast<const float4*>(bank), fused, cps, tpb,
                                    status, (cudaStream_t)stream);
}

}  // extern "C"
