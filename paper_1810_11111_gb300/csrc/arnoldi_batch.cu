// Arnoldi processes of many independent instances in one persistent launch
// per kernel class (see arnoldi_multi_kernel in sgk_arnoldi.cuh).
//
// Instances of a batch share (d, degree) classes; within a class every
// instance keeps its own launch arguments (slices, shared-memory layout,
// barrier counter, Krylov workspace), exactly those of its stand-alone
// persistent launch, so it computes bitwise the same basis and Hessenberg
// matrix.  The instances of a class are scheduled onto the device's CTAs by
// list scheduling: in one global order (most CTAs first, then longest), an
// instance takes the nb CTAs that become free first, and each of those CTAs
// appends (instance, slice) to its work list.  Every list follows the global
// order and every CTA of the launch is resident, so an instance's grid
// barriers only wait on CTAs that reach it.
#include <algorithm>
#include <array>
#include <memory>
#include <numeric>

#include "sgk_arnoldi.cuh"

namespace sgk_arn {
extern template void arn_multi_launch_k<2>(cudaStream_t, int, int, bool, const int*, const int2*, const void*,
                                           const ArnArgs*, const int*, int, size_t, size_t, int);
extern template void arn_multi_launch_k<3>(cudaStream_t, int, int, bool, const int*, const int2*, const void*,
                                           const ArnArgs*, const int*, int, size_t, size_t, int);
extern template void arn_multi_launch_k<4>(cudaStream_t, int, int, bool, const int*, const int2*, const void*,
                                           const ArnArgs*, const int*, int, size_t, size_t, int);
extern template void arn_multi_upload_ga<2>(const std::vector<const sgk_op*>&, DevBuf<unsigned char>&, cudaStream_t);
extern template void arn_multi_upload_ga<3>(const std::vector<const sgk_op*>&, DevBuf<unsigned char>&, cudaStream_t);
extern template void arn_multi_upload_ga<4>(const std::vector<const sgk_op*>&, DevBuf<unsigned char>&, cudaStream_t);
}  // namespace sgk_arn

using sgk_arn::ArnArgs;
using sgk_arn::ArnPrep;

ArnPrep arnoldi_prepare(sgk_ctx* ctx, const sgk_op* op, const PersistentWork& pw, const KrylovWork<double>& kw,
                        const double* v, int64_t n, int M);

namespace {

struct BatchClass {
    int d = 0, kp1 = 0, G = 0;
    bool df = false;
    size_t smem = 0;
    int grid = 0;
    DevBuf<int> item_off;
    DevBuf<int2> items;
    DevBuf<unsigned char> ga;
    DevBuf<ArnArgs> aa;
    DevBuf<int> nb;
};

// zero the barrier counter of every instance before a launch
__global__ void batch_bar_reset_kernel(unsigned* const* bars, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) bars[i][0] = 0u;
}

}  // namespace

struct ArnBatchPlan {
    std::vector<BatchClass> classes;
    DevBuf<unsigned*> bars;
    int nbars = 0;
    size_t smem_optin = 0;
    int num_sms = 0;
    int64_t max_items = 0;  // longest CTA work list (for the statistics)
};

bool arnoldi_batch_supports(const ArnJob& j) {
    const int d = j.op->idx->d, kp1 = j.op->idx->k + 1;
    return d >= 2 && d <= 4 && kp1 >= 2 && kp1 <= 4 && j.n >= 1 && j.n <= arnoldi_persistent_max_n(j.ctx);
}

ArnBatchPlan* arnoldi_batch_plan(const std::vector<ArnJob>& jobs, int num_sms, size_t smem_optin, cudaStream_t st) {
    std::unique_ptr<ArnBatchPlan> plan(new ArnBatchPlan());
    plan->smem_optin = smem_optin;
    plan->num_sms = num_sms;
    std::vector<ArnPrep> prep(jobs.size());
    std::vector<unsigned*> bars;
    for (size_t i = 0; i < jobs.size(); ++i) {
        const ArnJob& j = jobs[i];
        SGK_REQUIRE(arnoldi_batch_supports(j), SGK_EUNSUPPORTED, "batched Arnoldi: unsupported instance");
        prep[i] = arnoldi_prepare(j.ctx, j.op, j.pw, j.kw, j.v, j.n, j.M);
        // the batched kernels take 4 or 8 lanes per output
        prep[i].G = prep[i].G >= 8 ? 8 : 4;
        SGK_REQUIRE(prep[i].nb <= num_sms, SGK_EUNSUPPORTED, "batched Arnoldi: instance grid above the SM count");
        bars.push_back(j.pw.bar);
    }
    // classes: (d, k + 1, lanes, double-float)
    std::vector<std::vector<int>> cls;
    std::vector<std::array<int, 4>> keys;
    for (size_t i = 0; i < jobs.size(); ++i) {
        const std::array<int, 4> key = {prep[i].d, prep[i].kp1, prep[i].G, prep[i].a.df};
        auto it = std::find(keys.begin(), keys.end(), key);
        if (it == keys.end()) {
            keys.push_back(key);
            cls.emplace_back();
            it = keys.end() - 1;
        }
        cls[it - keys.begin()].push_back((int)i);
    }
    for (size_t c = 0; c < cls.size(); ++c) {
        std::vector<int>& mem = cls[c];
        // estimated duration of an instance: its longest slice's work per
        // step (gather entries of about 13 d per output, and 2 M for the
        // Gram-Schmidt passes) times M steps
        auto cost = [&](int i) {
            const ArnPrep& p = prep[i];
            return (double)p.a.M * (double)p.a.E * (13.0 * p.d + 2.0 * p.a.M);
        };
        std::stable_sort(mem.begin(), mem.end(), [&](int x, int y) {
            if (prep[x].nb != prep[y].nb) return prep[x].nb > prep[y].nb;
            return cost(x) > cost(y);
        });
        std::vector<double> avail(num_sms, 0.0);
        std::vector<std::vector<int2>> lists(num_sms);
        std::vector<int> order(num_sms);
        for (size_t li = 0; li < mem.size(); ++li) {
            const int i = mem[li];
            const int nb = prep[i].nb;
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return avail[x] < avail[y]; });
            std::sort(order.begin(), order.begin() + nb);  // the chosen CTAs in index order
            double start = 0.0;
            for (int b = 0; b < nb; ++b) start = std::max(start, avail[order[b]]);
            for (int b = 0; b < nb; ++b) {
                lists[order[b]].push_back(make_int2((int)li, b));
                avail[order[b]] = start + cost(i);
            }
        }
        // compact: only CTAs with work, in index order
        std::vector<int> off(1, 0);
        std::vector<int2> items;
        for (int b = 0; b < num_sms; ++b) {
            if (lists[b].empty()) continue;
            items.insert(items.end(), lists[b].begin(), lists[b].end());
            off.push_back((int)items.size());
            plan->max_items = std::max<int64_t>(plan->max_items, (int64_t)lists[b].size());
        }
        BatchClass& bc = *plan->classes.emplace(plan->classes.end());
        bc.d = keys[c][0];
        bc.kp1 = keys[c][1];
        bc.G = keys[c][2];
        bc.df = keys[c][3] != 0;
        bc.grid = (int)off.size() - 1;
        std::vector<ArnArgs> aa;
        std::vector<int> nbs;
        std::vector<const sgk_op*> ops;
        for (int i : mem) {
            aa.push_back(prep[i].a);
            nbs.push_back(prep[i].nb);
            ops.push_back(jobs[i].op);
            bc.smem = std::max(bc.smem, prep[i].smem);
        }
        bc.item_off.upload(off, st);
        bc.items.upload(items, st);
        bc.aa.upload(aa, st);
        bc.nb.upload(nbs, st);
        switch (bc.d) {
            case 2: sgk_arn::arn_multi_upload_ga<2>(ops, bc.ga, st); break;
            case 3: sgk_arn::arn_multi_upload_ga<3>(ops, bc.ga, st); break;
            default: sgk_arn::arn_multi_upload_ga<4>(ops, bc.ga, st); break;
        }
    }
    plan->bars.upload(bars, st);
    plan->nbars = (int)bars.size();
    SGK_CUDA_CHECK(cudaStreamSynchronize(st));  // the host vectors above go out of scope
    return plan.release();
}

int arnoldi_batch_launch(const ArnBatchPlan* plan, cudaStream_t st) {
    if (plan->nbars == 0) return 0;
    batch_bar_reset_kernel<<<(plan->nbars + 255) / 256, 256, 0, st>>>(plan->bars.p, plan->nbars);
    check_launch("batch_bar_reset");
    int launches = 1;
    for (const BatchClass& bc : plan->classes) {
        switch (bc.d) {
            case 2:
                sgk_arn::arn_multi_launch_k<2>(st, bc.kp1, bc.G, bc.df, bc.item_off.p, bc.items.p, bc.ga.p, bc.aa.p,
                                               bc.nb.p, bc.grid, bc.smem, plan->smem_optin, plan->num_sms);
                break;
            case 3:
                sgk_arn::arn_multi_launch_k<3>(st, bc.kp1, bc.G, bc.df, bc.item_off.p, bc.items.p, bc.ga.p, bc.aa.p,
                                               bc.nb.p, bc.grid, bc.smem, plan->smem_optin, plan->num_sms);
                break;
            default:
                sgk_arn::arn_multi_launch_k<4>(st, bc.kp1, bc.G, bc.df, bc.item_off.p, bc.items.p, bc.ga.p, bc.aa.p,
                                               bc.nb.p, bc.grid, bc.smem, plan->smem_optin, plan->num_sms);
                break;
        }
        check_launch("arnoldi_multi_kernel");
        ++launches;
    }
    return launches;
}

int arnoldi_batch_classes(const ArnBatchPlan* plan) { return plan ? (int)plan->classes.size() : 0; }

void arnoldi_batch_free(ArnBatchPlan* plan) { delete plan; }
