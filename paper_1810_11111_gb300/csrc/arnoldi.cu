// Persistent Arnoldi process for the Krylov approximation of exp(dt A) v
// (Section 3, eqs. krylov1-krylov3): gamma = ||v||, then M steps of matvec,
// classical Gram-Schmidt twice (CGS2) and normalisation, all in one
// cooperative launch.
//
// Each CTA owns a contiguous slice of the coefficient vector.  It computes
// the matvec outputs of its slice (gather form, sgk_gmv.h) and at once the
// partial inner products of that slice with the basis columns, so the
// matvec and the first projection need no barrier between them.  Two grid
// barriers per step publish (1) V^T w, (2) V^T w' together with ||w'||^2
// (the norm of w'' follows by Pythagoras; near breakdown a third barrier
// sums it explicitly); with the double-float matvec one more barrier at the
// start publishes the pairs of v / gamma for the first gathers (pairs of
// FP32 numbers cannot hold an unnormalised v of tiny magnitude).  The
// cross-CTA sums are exact: every CTA adds its
// partials, as 128-bit fixed-point integers, into integer accumulators with
// atomic adds, and after the barrier every CTA reads the same totals, so all
// CTAs hold bitwise equal h1, h2 and beta and take the same breakdown
// decision without another barrier; the results do not depend on the order
// in which CTAs arrive.  The next matvec gathers the unnormalised w' and
// forms A v_{j+1} = (A w' - Z h2) / beta from the stored raw outputs Z; the
// two w buffers alternate so that those gathers never race with the writes
// of the next step.  Accumulator sets rotate over three buffers for the same
// reason.
//
// Barriers are counters in global memory with a bounded wait: a CTA that
// waits longer than the limit sets an error flag and returns, and every
// other CTA sees the flag in its own wait and returns too; the host reports
// SGK_ETIMEOUT.  The cooperative launch makes every CTA resident at once.
#include <cmath>
#include <cstdlib>

#include "sgk_arnoldi.cuh"

namespace sgk_arn {
extern template void arn_launch_k<1>(sgk_ctx*, const sgk_op*, const ArnArgs&, int, size_t, int);
extern template void arn_launch_k<2>(sgk_ctx*, const sgk_op*, const ArnArgs&, int, size_t, int);
extern template void arn_launch_k<3>(sgk_ctx*, const sgk_op*, const ArnArgs&, int, size_t, int);
extern template void arn_launch_k<4>(sgk_ctx*, const sgk_op*, const ArnArgs&, int, size_t, int);
extern template void arn_launch_k<5>(sgk_ctx*, const sgk_op*, const ArnArgs&, int, size_t, int);
extern template void arn_launch_k<6>(sgk_ctx*, const sgk_op*, const ArnArgs&, int, size_t, int);
}  // namespace sgk_arn

using sgk_arn::ArnArgs;
using sgk_arn::ArnPrep;
using sgk_arn::PT;
using sgk_arn::arn_launch_k;

static int persistent_ctas(const sgk_ctx* ctx) {
    return ctx->persist_ctas > 0 ? std::min(ctx->persist_ctas, ctx->num_sms) : ctx->num_sms;
}

int arnoldi_persistent_ctas(const sgk_ctx* ctx) { return persistent_ctas(ctx); }

int64_t arnoldi_persistent_max_n(const sgk_ctx* ctx) {
    // two slices of w are staged in shared memory: at most 12 K doubles each
    return (int64_t)persistent_ctas(ctx) * 12 * 1024;
}

size_t arnoldi_persistent_pbuf_size(const sgk_ctx* ctx, int M) {
    (void)M;
    // per-CTA norm partials, then the three fixed-point accumulator sets
    return (size_t)ctx->num_sms + 3 * sgk_arn::FX_SET;
}

static size_t smem_budget(const sgk_ctx* ctx) {
    // the kernel's static shared memory stays below 13 KB
    return ctx->smem_optin > 16 * 1024 ? ctx->smem_optin - 13 * 1024 : 32 * 1024;
}

std::vector<int64_t> arnoldi_balanced_bounds(const sgk_ctx* ctx, const sgk_op* op, int M, int64_t* E,
                                             int64_t* list_ent) {
    const int nb = persistent_ctas(ctx);
    const int64_t n = op->idx->dof;
    const int d = op->idx->d;
    const int64_t per = PT / 8;  // outputs of one matvec pass at 8 lanes each
    // no more matvec passes than equal slices need (a pass costs about as
    // much as 8 K gather entries)
    const int64_t cap_len = std::min<int64_t>(((n + nb - 1) / nb + per - 1) / per * per, 12 * 1024);
    // shared memory left for the entries with the longest slice's w, V, Z
    // and entry offsets staged
    const size_t fixed = sizeof(double) * (2 * (size_t)cap_len + 2 * (size_t)(M + 1) * (size_t)(cap_len | 1)) +
                         sgk_arn::arn_eoff_bytes((int)cap_len, d);
    const size_t budget = smem_budget(ctx);
    int64_t cap_ent = (op->gmv_ecnt_host.empty() || fixed >= budget) ? (int64_t(1) << 40)
                                                                      : (int64_t)((budget - fixed) / sizeof(int2));
    std::vector<int64_t> b = arnoldi_slice_bounds(op, nb, 2 * M, cap_len, cap_ent);
    *E = 0;
    *list_ent = 0;
    for (size_t i = 0; i + 1 < b.size(); ++i) {
        *E = std::max<int64_t>(*E, b[i + 1] - b[i]);
        if (!op->gmv_ecnt_host.empty()) {
            int64_t e = 0;
            for (int64_t g = b[i]; g < b[i + 1]; ++g) e += op->gmv_ecnt_host[g];
            *list_ent = std::max(*list_ent, e);
        }
    }
    return b;
}

static size_t loc_bytes(int d) {
    switch (d) {
        case 1: return sizeof(GmvLoc<1>);
        case 2: return sizeof(GmvLoc<2>);
        case 3: return sizeof(GmvLoc<3>);
        case 4: return sizeof(GmvLoc<4>);
        case 5: return sizeof(GmvLoc<5>);
        default: return sizeof(GmvLoc<6>);
    }
}

// The launch arguments of one Arnoldi process (shared memory layout, slices,
// fixed-point scales, arithmetic) for the persistent kernel on ctx's grid.
ArnPrep arnoldi_prepare(sgk_ctx* ctx, const sgk_op* op, const PersistentWork& pw, const KrylovWork<double>& kw,
                        const double* v, int64_t n, int M) {
    SGK_REQUIRE(n >= 1 && n <= arnoldi_persistent_max_n(ctx), SGK_EUNSUPPORTED, "persistent Arnoldi: n too large");
    SGK_REQUIRE(M >= 1 && M <= SGK_MAX_KRYLOV, SGK_EINVAL, "persistent Arnoldi: bad M");
    const int nb = persistent_ctas(ctx);
    // the fixed-point limb sums hold one term below 2^56 per CTA
    SGK_REQUIRE(nb <= 255, SGK_EUNSUPPORTED, "persistent Arnoldi: more than 255 CTAs");
    const int64_t E = pw.bounds ? pw.E : (n + nb - 1) / nb;
    SGK_REQUIRE(E >= 1 && E <= 12 * 1024, SGK_EUNSUPPORTED, "persistent Arnoldi: slice too long");
    // lanes per output in the matvec: the autotuned value, else eight (the
    // gathers are latency-bound; more lanes keep more of them in flight)
    const int G = pw.G > 0 ? pw.G : 8;
    ArnArgs a;
    a.n = n;
    a.M = M;
    a.E = (int)E;
    a.v = v;
    a.V = kw.V;
    a.w0 = kw.w;
    a.w1 = pw.w_alt;
    a.Z = pw.Z;
    a.H = kw.H;
    a.pbuf = pw.pbuf;
    a.acc = reinterpret_cast<unsigned long long*>(pw.pbuf + ctx->num_sms);
    // fixed-point scales from the bound ||A v|| <= ||A|| for ||v|| = 1:
    // |partial| <= 2^(e - 1) with e = ceil(log2 ||A||) + 1, entered as
    // floor(p 2^(110 - e)), so |P| < 2^110; the squared norm likewise with 2e
    {
        const double an = op->anorm > 0.0 ? op->anorm : 1.0;
        const int e = std::min(400, std::max(-400, (int)std::ceil(std::log2(an)) + 1));
        a.sc_h = std::ldexp(1.0, 46 - e);
        a.isc_h = std::ldexp(1.0, e - 110);
        a.sc_n = std::ldexp(1.0, 46 - 2 * e);
        a.isc_n = std::ldexp(1.0, 2 * e - 110);
    }
    a.bar = pw.bar;
    // failure injection on the host: with SGK_TEST_BARRIER_STALL set, every
    // barrier waits for one arrival more than the grid has, so the bounded
    // waits run out and the launch ends with the error flag set
    a.bar_extra = std::getenv("SGK_TEST_BARRIER_STALL") ? 1u : 0u;
    a.ks = kw.ks;
    a.bounds = pw.bounds;
    // shared memory: the slice of w always; the slices of V and Z (all
    // M + 1 columns) and the slice's pre-located gathers (else the located
    // rows of its outputs) when they fit, which turns the Gram-Schmidt,
    // correction and gather-address loads into shared loads (an acquire at a
    // grid barrier empties L1)
    const int d = op->idx->d;
    int64_t list_ent = pw.bounds ? pw.list_ent : 0;
    if (!pw.bounds && !op->gmv_ecnt_host.empty())
        for (int bb = 0; bb < nb; ++bb) {
            int64_t e = 0;
            for (int64_t g = std::min<int64_t>(n, bb * E); g < std::min<int64_t>(n, (bb + 1) * E); ++g)
                e += op->gmv_ecnt_host[g];
            list_ent = std::max(list_ent, e);
        }
    const bool has_list = !op->gmv_ecnt_host.empty() && op->gmv_ent.p != nullptr;
    const size_t budget = smem_budget(ctx);
    const size_t ws = sizeof(double) * 2 * (size_t)E;  // two staged slices of w
    const size_t vz = sizeof(double) * 2 * (size_t)(M + 1) * (size_t)(E | 1);  // odd column stride
    const size_t lb = loc_bytes(d) * (size_t)E;
    const size_t lst = sgk_arn::arn_eoff_bytes((int)E, d) + sizeof(int2) * (size_t)std::max<int64_t>(list_ent, 1);
    a.eoff = has_list ? op->gmv_eoff.p : nullptr;
    a.ent = has_list ? op->gmv_ent.p : nullptr;
    a.smem_vz = 0;
    a.smem_loc = 0;
    a.list_cap = 0;
    if (has_list && ws + vz + lst <= budget) {
        a.smem_vz = 1;
        a.list_cap = (int)std::max<int64_t>(list_ent, 1);
    } else if (has_list && ws + lst <= budget) {
        a.list_cap = (int)std::max<int64_t>(list_ent, 1);
    } else {
        a.smem_vz = ws + vz <= budget;
        a.smem_loc = ws + (a.smem_vz ? vz : 0) + lb <= budget;
    }
    const size_t smem = ws + (a.smem_vz ? vz : 0) + (a.list_cap ? lst : 0) + (a.smem_loc ? lb : 0);
    // mixed precision: the matvec in double-float arithmetic (~1e-14
    // relative; FP64 issue on this part is 1/64 of FP32), with the gather lists
    a.cvk2 = op->gmv_cvk2.p;
    a.df = ctx->precision == SGK_MIXED && a.list_cap > 0 && op->gmv_cvk2.p != nullptr;
    ArnPrep out;
    out.a = a;
    out.smem = smem;
    out.nb = nb;
    out.G = G;
    out.d = d;
    out.kp1 = op->idx->k + 1;
    return out;
}

void arnoldi_persistent(sgk_ctx* ctx, const sgk_op* op, const PersistentWork& pw, const KrylovWork<double>& kw,
                        const double* v, int64_t n, int M) {
    const ArnPrep p = arnoldi_prepare(ctx, op, pw, kw, v, n, M);
    const ArnArgs& a = p.a;
    const int nb = p.nb, G = p.G;
    const size_t smem = p.smem;
    KTimer kt(ctx, KC_KRYLOV);
    SGK_CUDA_CHECK(cudaMemsetAsync(pw.bar, 0, sizeof(unsigned), ctx->stream));
    switch (op->idx->d) {
        case 1: arn_launch_k<1>(ctx, op, a, nb, smem, G); break;
        case 2: arn_launch_k<2>(ctx, op, a, nb, smem, G); break;
        case 3: arn_launch_k<3>(ctx, op, a, nb, smem, G); break;
        case 4: arn_launch_k<4>(ctx, op, a, nb, smem, G); break;
        case 5: arn_launch_k<5>(ctx, op, a, nb, smem, G); break;
        case 6: arn_launch_k<6>(ctx, op, a, nb, smem, G); break;
        default: throw SgkError{SGK_EUNSUPPORTED, "persistent Arnoldi: d must be 1..6"};
    }
    check_launch("arnoldi_kernel");
    count_launch(ctx);
}

namespace {

// Deterministic test vector for the tuning runs (no method arithmetic):
// x_i = frac(i * golden ratio) - 1/2.
__global__ void tune_fill_kernel(double* x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double t = (double)(i + 1) * 0.6180339887498949;
        x[i] = (t - floor(t)) - 0.5;
    }
}

}  // namespace

int arnoldi_autotune(sgk_ctx* ctx, const sgk_op* op, PersistentWork pw, const KrylovWork<double>& kw, double* scratch,
                     int64_t n, int M) {
    // candidate lane counts per output, each timed (best of three) on full
    // Arnoldi processes of a fixed vector after a warm-up run; ties keep the
    // larger G
    tune_fill_kernel<<<std::min<int64_t>((n + 255) / 256, 1024), 256, 0, ctx->stream>>>(scratch, n);
    check_launch("tune_fill");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SGK_CUDA_CHECK(cudaEventCreate(&e0));
    SGK_CUDA_CHECK(cudaEventCreate(&e1));
    int best = 8;
    float best_ms = 1e30f;
    try {
        for (int G : {8, 4, 2}) {
            pw.G = G;
            arnoldi_persistent(ctx, op, pw, kw, scratch, n, M);
            float ms = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                SGK_CUDA_CHECK(cudaEventRecord(e0, ctx->stream));
                arnoldi_persistent(ctx, op, pw, kw, scratch, n, M);
                SGK_CUDA_CHECK(cudaEventRecord(e1, ctx->stream));
                SGK_CUDA_CHECK(cudaEventSynchronize(e1));
                float t = 0.f;
                SGK_CUDA_CHECK(cudaEventElapsedTime(&t, e0, e1));
                ms = std::min(ms, t);
            }
            if (ms < 0.97f * best_ms) {
                best_ms = ms;
                best = G;
            }
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}
