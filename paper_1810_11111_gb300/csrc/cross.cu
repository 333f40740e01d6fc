// Mixed-derivative terms of the SIPG operator for a constant SPD diffusion
// tensor K with off-diagonal entries (Section 2.1, the bilinear form B with
// k grad u . grad v and its face terms; eq. sp3 for the fluxes).
//
// For a pair of directions i < j the form adds -K_ij B_ij with, in 1D
// factors (test index first; the first factor acts along i, the second
// along j),
//   B_ij = P x P^T + P^T x P - E x P^T - P^T x E - E^T x P - P x E^T
//        = Q x P^T + P^T x Q - E^T x P - P x E^T,   Q = P - E,
// P[a][b] = sum over finest cells of int v_a' v_b and E[a][b] = sum over
// faces of [v_a] {v_b} (tables.cpp).  The sparse-grid operator is the full
// tensor one restricted to the index set (Galerkin), so output a collects,
// per pair and term X x Y, sum_{b_i, b_j} X[a_i][b_i] Y[a_j][b_j] x[b] over
// the b that agree with a outside i, j and lie in the index set: l(b_i) +
// l(b_j) <= N - sum_{m != i, j} l_m.  The rows of X and Y are stored sorted
// by column (so by level) with their lengths truncated per level, as for
// the diagonal part; the block offsets of the tuples reached by changing
// the levels of i and j are tabulated per (tuple, pair) on the host.
//
// The kernel adds these terms to y after the diagonal gather (gmv_kernel):
// one thread per output, the two factors' rows walked as a sum-factorised
// double loop.
#include <algorithm>
#include <cmath>
#include <map>

#include "sgk_internal.h"

namespace {

constexpr int XT = 4;  // stored 1D matrices: Q, P^T, E^T, P

template <typename T>
__global__ void __launch_bounds__(256) cross_kernel(int64_t dof, int d, int N, int kp1, int64_t ntuples,
                                                    const int32_t* __restrict__ levels,
                                                    const int64_t* __restrict__ offsets, int npairs,
                                                    const int* __restrict__ pair_ij, const double* __restrict__ kij,
                                                    const int* __restrict__ xptr, const int* __restrict__ xcol,
                                                    const T* __restrict__ xval, const int* __restrict__ xrlen,
                                                    const int64_t* __restrict__ grp, const int64_t* __restrict__ xoff,
                                                    const T* __restrict__ x, T* __restrict__ y) {
    const int H = kp1 << N;
    const int nl = N + 1;
    // the four terms: (X along i, Y along j, sign)
    const int tx[4] = {0, 1, 2, 3}, ty[4] = {1, 0, 3, 2};
    const T sg[4] = {T(1), T(1), T(-1), T(-1)};
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < dof; g += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = ntuples;  // offsets[lo] <= g < offsets[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) / 2;
            if (offsets[mid] <= g) lo = mid;
            else hi = mid;
        }
        int l[SGK_MAX_DIM], t[SGK_MAX_DIM], a[SGK_MAX_DIM];
        int64_t loc = g - offsets[lo];
        int lsum = 0;
        for (int m = d - 1; m >= 0; --m) {
            l[m] = levels[lo * d + m];
            const int n_l = l[m] == 0 ? kp1 : kp1 << (l[m] - 1);
            t[m] = (int)(loc % n_l);
            loc /= n_l;
            a[m] = (l[m] == 0 ? 0 : kp1 << (l[m] - 1)) + t[m];
            lsum += l[m];
        }
        T acc_all = T(0);
        for (int p = 0; p < npairs; ++p) {
            const int i = pair_ij[2 * p], j = pair_ij[2 * p + 1];
            const int L = N - (lsum - l[i] - l[j]);
            const int64_t* offs = xoff + grp[lo * npairs + p];
            // strides of the block layout (last dimension fastest) with the
            // extents of i and j left out: a position is
            // (sum over m of t_m stride_m) with stride_m = prod_{m' > m} n_m'
            T acc = T(0);
            for (int term = 0; term < 4; ++term) {
                const int X = tx[term], Y = ty[term];
                const int* px = xptr + (size_t)X * (H + 1);
                const int* py = xptr + (size_t)Y * (H + 1);
                const int xb = px[a[i]], xe = xb + xrlen[((size_t)X * H + a[i]) * nl + L];
                T tacc = T(0);
                for (int e = xb; e < xe; ++e) {
                    const int bi = xcol[e];
                    const int qi = bi / kp1;
                    const int li = qi == 0 ? 0 : 32 - __clz(qi);
                    const int Lj = L - li;
                    const int yb = py[a[j]], ye = yb + xrlen[((size_t)Y * H + a[j]) * nl + Lj];
                    const int ti = bi - (li == 0 ? 0 : kp1 << (li - 1));
                    T inner = T(0);
                    for (int f = yb; f < ye; ++f) {
                        const int bj = xcol[f];
                        const int qj = bj / kp1;
                        const int lj = qj == 0 ? 0 : 32 - __clz(qj);
                        const int tj = bj - (lj == 0 ? 0 : kp1 << (lj - 1));
                        // position of b in the block of (l with l_i = li, l_j = lj)
                        int64_t pos = 0;
                        for (int m = 0; m < d; ++m) {
                            const int lm = m == i ? li : (m == j ? lj : l[m]);
                            const int n_m = lm == 0 ? kp1 : kp1 << (lm - 1);
                            pos = pos * n_m + (m == i ? ti : (m == j ? tj : t[m]));
                        }
                        inner += xval[f] * x[offs[li * (L + 1) + lj] + pos];
                    }
                    tacc += xval[e] * inner;
                }
                acc += sg[term] * tacc;
            }
            acc_all += (T)kij[p] * acc;
        }
        y[g] -= acc_all;
    }
}

}  // namespace

// Host tables of the mixed-derivative terms of op for the tensor K (d x d,
// row-major, symmetric); no-op when K is diagonal.
void build_cross_tables(sgk_op* op, const double* K) {
    const sgk_index* idx = op->idx;
    const int d = idx->d, N = idx->n, kp1 = idx->k + 1, H = op->H, nl = N + 1;
    std::vector<int> pij;
    std::vector<double> kij;
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j)
            if (K[i * d + j] != 0.0) {
                pij.push_back(i);
                pij.push_back(j);
                kij.push_back(K[i * d + j]);
            }
    op->npairs = (int)kij.size();
    if (op->npairs == 0) return;
    Tables1D tab;
    build_transform_tables(N, idx->k, tab);
    std::vector<double> P, E;
    build_cross_hier(tab, op->bc, P, E);
    // dense 1D factors: Q = P - E, P^T, E^T, P; entries below 1e-13 of a
    // matrix's largest are rounding residue of the change of basis
    std::vector<double> Xd((size_t)XT * H * H);
    for (int a = 0; a < H; ++a)
        for (int b = 0; b < H; ++b) {
            const size_t ab = (size_t)a * H + b, ba = (size_t)b * H + a;
            Xd[0 * (size_t)H * H + ab] = P[ab] - E[ab];
            Xd[1 * (size_t)H * H + ab] = P[ba];
            Xd[2 * (size_t)H * H + ab] = E[ba];
            Xd[3 * (size_t)H * H + ab] = P[ab];
        }
    std::vector<int> ptr, col, rl((size_t)XT * H * nl);
    std::vector<double> val;
    ptr.reserve((size_t)XT * (H + 1));
    for (int X = 0; X < XT; ++X) {
        double mx = 0.0;
        for (size_t e = 0; e < (size_t)H * H; ++e) mx = std::max(mx, std::abs(Xd[(size_t)X * H * H + e]));
        const int base = (int)col.size();
        for (int a = 0; a < H; ++a) {
            ptr.push_back((int)col.size());
            for (int b = 0; b < H; ++b) {
                const double v = Xd[(size_t)X * H * H + (size_t)a * H + b];
                if (std::abs(v) > 1e-13 * mx) {
                    col.push_back(b);
                    val.push_back(v);
                }
            }
        }
        ptr.push_back((int)col.size());
        (void)base;
        // truncated lengths: entries of row a with column < (k+1) 2^L
        for (int a = 0; a < H; ++a) {
            const int rb = ptr[(size_t)X * (H + 1) + a], re = ptr[(size_t)X * (H + 1) + a + 1];
            for (int L = 0; L < nl; ++L) {
                const int lim = kp1 << L;
                int c = 0;
                for (int e = rb; e < re && col[e] < lim; ++e) ++c;
                rl[((size_t)X * H + a) * nl + L] = c;
            }
        }
    }
    // block offsets of the tuples reached from each tuple by changing the
    // levels of i and j, per pair: one table per (pair, other levels), shared
    // by the tuples with those other levels; -1 outside the index set
    const int64_t nt = idx->ntuples;
    std::vector<int64_t> grp((size_t)nt * op->npairs), off;
    for (int p = 0; p < op->npairs; ++p) {
        const int i = pij[2 * p], j = pij[2 * p + 1];
        std::map<std::vector<int>, int64_t> seen;
        for (int64_t tu = 0; tu < nt; ++tu) {
            std::vector<int> l(idx->levels.begin() + tu * d, idx->levels.begin() + (tu + 1) * d);
            std::vector<int> rest;
            int rs = 0;
            for (int m = 0; m < d; ++m)
                if (m != i && m != j) {
                    rest.push_back(l[m]);
                    rs += l[m];
                }
            auto it = seen.find(rest);
            if (it == seen.end()) {
                const int L = N - rs;
                const int64_t b0 = (int64_t)off.size();
                for (int li = 0; li <= L; ++li)
                    for (int lj = 0; lj <= L; ++lj) {
                        if (li + lj > L) {
                            off.push_back(-1);
                            continue;
                        }
                        std::vector<int> lt = l;
                        lt[i] = li;
                        lt[j] = lj;
                        off.push_back(idx->offsets[tuple_rank(lt, N)]);
                    }
                it = seen.emplace(rest, b0).first;
            }
            grp[(size_t)tu * op->npairs + p] = it->second;
        }
    }
    cudaStream_t s = op->ctx->stream;
    op->x_pairs.upload(pij, s);
    op->x_kij.upload(kij, s);
    op->x_ptr.upload(ptr, s);
    op->x_col.upload(col, s);
    op->x_val.upload(val, s);
    std::vector<float> valf(val.begin(), val.end());
    op->x_valf.upload(valf, s);
    op->x_rlen.upload(rl, s);
    op->x_grp.upload(grp, s);
    op->x_off.upload(off, s);
    // multiply-adds of one application: per output and pair, the four terms'
    // truncated row products (counted on the host for the benchmarks)
    SGK_CUDA_CHECK(cudaStreamSynchronize(s));
    for (int X = 0; X < XT; ++X) op->x_nnz += ptr[(size_t)X * (H + 1) + H] - ptr[(size_t)X * (H + 1)];
}

template <typename T>
void op_cross_matvec(const sgk_op* op, const T* x, T* y) {
    if (op->npairs == 0 || op->idx->dof == 0) return;
    const sgk_index* idx = op->idx;
    sgk_ctx* ctx = op->ctx;
    const T* vals = sizeof(T) == 8 ? reinterpret_cast<const T*>(op->x_val.p) : reinterpret_cast<const T*>(op->x_valf.p);
    const int grid = (int)std::min<int64_t>((idx->dof + 255) / 256, (int64_t)ctx->num_sms * 8);
    KTimer kt(ctx, KC_MATVEC);
    cross_kernel<T><<<grid, 256, 0, ctx->stream>>>(idx->dof, idx->d, idx->n, idx->k + 1, idx->ntuples,
                                                   idx->d_levels.p, idx->d_offsets.p, op->npairs, op->x_pairs.p,
                                                   op->x_kij.p, op->x_ptr.p, op->x_col.p, vals, op->x_rlen.p,
                                                   op->x_grp.p, op->x_off.p, x, y);
    check_launch("cross_kernel");
    count_launch(ctx);
}

template void op_cross_matvec<double>(const sgk_op*, const double*, double*);
template void op_cross_matvec<float>(const sgk_op*, const float*, float*);
