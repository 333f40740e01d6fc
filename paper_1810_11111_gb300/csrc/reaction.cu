// Reaction term F(U) = (int f(u_h) v_a dx)_a and its Jacobian product
// J_F(U) w = (int f'(u_h) w_h v_a dx)_a by finest-grid Gauss quadrature
// (Section 4: u_h is reconstructed at the Gauss points of the finest mesh and
// the integral is evaluated by quadrature; Section 5 calls this the most
// costly part).
//
// Pipeline per species (all on the device):
//   1. forward change of basis, one direction at a time (fiber engine, FWD):
//      sparse hierarchical coefficients -> finest-cell Legendre coefficients
//      on the full grid ((k+1) 2^N)^d.  After direction i the array holds
//      blocks over the level tuples of directions i+1..d-1, each with
//      directions 0..i already full;
//   2. cell kernel: per finest cell, Legendre -> q^d Gauss points
//      (sum-factorised, one direction at a time), pointwise f (species
//      coupled) or f' w, times the quadrature weights, back to the (k+1)^d
//      Legendre moments;
//   3. backward change of basis (fiber engine, BWD, transpose of step 1)
//      back to the sparse index set.
// q = ceil((p k + k + 1)/2) for total reaction degree p makes F the exact L2
// projection of f(u_h) onto the sparse-grid space.
#include <algorithm>
#include <cmath>

#include "sgk_dfloat.h"
#include "sgk_quad.h"

namespace {

template <typename T>
struct CellParams {
    int d, kp1, q, ncell1, H, cpb, maxstage, nspecies;
    long long ncells;
    long long Hpow[SGK_MAX_DIM];
    const T* u[SGK_MAX_SPECIES];
    const T* w[SGK_MAX_SPECIES];
    T* out[SGK_MAX_SPECIES];
    const T* B;   // q x kp1
    const T* w1;  // q
    ReactionDev rx;
};

__host__ __device__ __forceinline__ int ipow(int b, int e) {
    int r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

template <typename T>
__device__ __forceinline__ T powi(T x, int e) {
    T r = T(1);
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

template <typename T, int JAC>
__global__ void __launch_bounds__(256) cell_kernel(const CellParams<T> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int S = p.nspecies;
    const int nsets = JAC ? 2 * S : S;
    const int kp1 = p.kp1, q = p.q, d = p.d, ms = p.maxstage;
    const int ncoef = ipow(kp1, d), npts = ipow(q, d);
    const long long set_stride = 2LL * p.cpb * ms;
    for (long long cell0 = blockIdx.x * (long long)p.cpb; cell0 < p.ncells; cell0 += (long long)gridDim.x * p.cpb) {
        const int ncb = (int)min((long long)p.cpb, p.ncells - cell0);
        // 1. gather (k+1)^d Legendre coefficients of each cell
        for (int set = 0; set < nsets; ++set) {
            const T* src = set < S ? p.u[set] : p.w[set - S];
            T* b = sm + set * set_stride;
            for (int e = threadIdx.x; e < ncb * ncoef; e += blockDim.x) {
                const int rl = e % kp1;
                const int t = e / kp1;
                const int cell = t % ncb;
                const int rpre = t / ncb;
                long long lin = cell0 + cell;
                long long addr = 0;
                int rr = rpre * kp1 + rl;
                for (int m = d - 1; m >= 0; --m) {
                    const int c = (int)(lin % p.ncell1);
                    lin /= p.ncell1;
                    const int r = rr % kp1;
                    rr /= kp1;
                    addr += (long long)(c * kp1 + r) * p.Hpow[d - 1 - m];
                }
                b[cell * ms + rpre * kp1 + rl] = src[addr];
            }
        }
        __syncthreads();
        // 2. forward contraction r -> g, direction d-1 first
        int cur = 0;
        for (int m = d - 1; m >= 0; --m) {
            const int suf = ipow(q, d - 1 - m);
            const int nout = ipow(kp1, m) * q * suf;
            for (int set = 0; set < nsets; ++set) {
                const T* in = sm + set * set_stride + cur * p.cpb * ms;
                T* out = sm + set * set_stride + (cur ^ 1) * p.cpb * ms;
                for (int e = threadIdx.x; e < ncb * nout; e += blockDim.x) {
                    const int cell = e / nout;
                    const int rem = e - cell * nout;
                    const int s_ = rem % suf;
                    const int t = rem / suf;
                    const int g = t % q;
                    const int P = t / q;
                    const T* ip = in + cell * ms + (P * kp1) * suf + s_;
                    T acc = T(0);
                    for (int r = 0; r < kp1; ++r) acc += p.B[g * kp1 + r] * ip[r * suf];
                    out[cell * ms + rem] = acc;
                }
            }
            cur ^= 1;
            __syncthreads();
        }
        // 3. pointwise f(u) or f'(u) w, times the tensor quadrature weight
        for (int e = threadIdx.x; e < ncb * npts; e += blockDim.x) {
            const int cell = e / npts;
            const int g = e - cell * npts;
            T wt = T(1);
            int gg = g;
            for (int m = 0; m < d; ++m) {
                wt *= p.w1[gg % q];
                gg /= q;
            }
            T uv[SGK_MAX_SPECIES], wv[SGK_MAX_SPECIES], res[SGK_MAX_SPECIES];
            for (int s = 0; s < S; ++s) {
                uv[s] = sm[s * set_stride + cur * p.cpb * ms + cell * ms + g];
                if (JAC) wv[s] = sm[(S + s) * set_stride + cur * p.cpb * ms + cell * ms + g];
                res[s] = T(0);
            }
            for (int mo = 0; mo < p.rx.nmono; ++mo) {
                const int s = p.rx.species[mo];
                const T c = T(p.rx.coef[mo]);
                if (!JAC) {
                    T t = c;
                    for (int r = 0; r < S; ++r) t *= powi(uv[r], p.rx.exps[mo][r]);
                    res[s] += t;
                } else {
                    for (int r = 0; r < S; ++r) {
                        const int er = p.rx.exps[mo][r];
                        if (er == 0) continue;
                        T t = c * T(er) * wv[r];
                        for (int r2 = 0; r2 < S; ++r2) t *= powi(uv[r2], p.rx.exps[mo][r2] - (r2 == r ? 1 : 0));
                        res[s] += t;
                    }
                }
            }
            for (int s = 0; s < S; ++s) sm[s * set_stride + (cur ^ 1) * p.cpb * ms + cell * ms + g] = wt * res[s];
        }
        __syncthreads();
        cur ^= 1;
        // 4. backward contraction g -> r (transpose), direction d-1 first
        for (int m = d - 1; m >= 0; --m) {
            const int suf = ipow(kp1, d - 1 - m);
            const int nout = ipow(q, m) * kp1 * suf;
            for (int s = 0; s < S; ++s) {
                const T* in = sm + s * set_stride + cur * p.cpb * ms;
                T* out = sm + s * set_stride + (cur ^ 1) * p.cpb * ms;
                for (int e = threadIdx.x; e < ncb * nout; e += blockDim.x) {
                    const int cell = e / nout;
                    const int rem = e - cell * nout;
                    const int s_ = rem % suf;
                    const int t = rem / suf;
                    const int r = t % kp1;
                    const int P = t / kp1;
                    const T* ip = in + cell * ms + (P * q) * suf + s_;
                    T acc = T(0);
                    for (int g = 0; g < q; ++g) acc += p.B[g * kp1 + r] * ip[g * suf];
                    out[cell * ms + rem] = acc;
                }
            }
            cur ^= 1;
            __syncthreads();
        }
        // 5. scatter the moments
        for (int s = 0; s < S; ++s) {
            const T* b = sm + s * set_stride + cur * p.cpb * ms;
            T* dst = p.out[s];
            for (int e = threadIdx.x; e < ncb * ncoef; e += blockDim.x) {
                const int rl = e % kp1;
                const int t = e / kp1;
                const int cell = t % ncb;
                const int rpre = t / ncb;
                long long lin = cell0 + cell;
                long long addr = 0;
                int rr = rpre * kp1 + rl;
                for (int m = d - 1; m >= 0; --m) {
                    const int c = (int)(lin % p.ncell1);
                    lin /= p.ncell1;
                    const int r = rr % kp1;
                    rr /= kp1;
                    addr += (long long)(c * kp1 + r) * p.Hpow[d - 1 - m];
                }
                dst[addr] = b[cell * ms + rpre * kp1 + rl];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------- projection ---

// Finest-cell Legendre moments of g(2 pi w x): out[t][m][c (k+1) + r].
__global__ void proj_fine_kernel(int nterms, int d, int N, int kp1, const int* __restrict__ wavenum,
                                 const int* __restrict__ kind, const double* __restrict__ xg,
                                 const double* __restrict__ wg, int nq, double* __restrict__ out) {
    const int H = kp1 << N;
    const long long total = (long long)nterms * d * H;
    const double h = ldexp(1.0, -N);
    const double pi = 3.141592653589793;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i % H);
        const long long tm = i / H;
        const int c = y / kp1, r = y % kp1;
        const int wn = wavenum[tm];
        const int kd = kind[tm];
        double acc = 0.0;
        for (int g = 0; g < nq; ++g) {
            const double xi = xg[g];
            const double x = (c + 0.5 * (xi + 1.0)) * h;
            // P_r(xi) by recurrence
            double p0 = 1.0, p1 = xi, pr = 1.0;
            if (r == 1) pr = xi;
            for (int j = 1; j < r; ++j) {
                const double p2 = ((2 * j + 1) * xi * p1 - j * p0) / (j + 1);
                p0 = p1;
                p1 = p2;
                pr = p2;
            }
            const double L = sqrt(2.0 * r + 1.0) * pr / sqrt(h);
            const double arg = 2.0 * pi * wn * x;
            const double gv = kd == 0 ? sin(arg) : cos(arg);
            acc += 0.5 * h * wg[g] * gv * L;
        }
        out[i] = acc;
    }
}

// Hierarchical 1D projections: out[t][m][a] = sum_y T^T[a][y] fine[t][m][y].
__global__ void proj_hier_kernel(long long nvec, int H, const int* __restrict__ tp, const int* __restrict__ tc,
                                 const double* __restrict__ tv, const double* __restrict__ fine,
                                 double* __restrict__ out) {
    const long long total = nvec * H;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(i % H);
        const long long v = i / H;
        double acc = 0.0;
        for (int e = tp[a]; e < tp[a + 1]; ++e) acc += tv[e] * fine[v * H + tc[e]];
        out[i] = acc;
    }
}

// U[e] = sum_t amp_t prod_m P1[t][m][a_m(e)] (+ c0 on the constant function).
__global__ void proj_product_kernel(long long dof, int d, int kp1, int H, long long ntuples,
                                    const int* __restrict__ levels, const long long* __restrict__ offsets, int nterms,
                                    const double* __restrict__ amp, const double* __restrict__ P1, double c0,
                                    double* __restrict__ U) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < dof;
         e += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = ntuples;  // offsets[lo] <= e < offsets[hi]
        while (hi - lo > 1) {
            const long long mid = (lo + hi) / 2;
            if (offsets[mid] <= e) lo = mid;
            else hi = mid;
        }
        long long loc = e - offsets[lo];
        int a[SGK_MAX_DIM];
        for (int m = d - 1; m >= 0; --m) {
            const int l = levels[lo * d + m];
            const int nl = l == 0 ? kp1 : kp1 << (l - 1);
            const int t = (int)(loc % nl);
            loc /= nl;
            a[m] = (l == 0 ? 0 : kp1 << (l - 1)) + t;
        }
        double acc = e == 0 ? c0 : 0.0;
        for (int t = 0; t < nterms; ++t) {
            double prod = amp[t];
            for (int m = 0; m < d; ++m) prod *= P1[((long long)t * d + m) * H + a[m]];
            acc += prod;
        }
        U[e] = acc;
    }
}

// b[e] = sum_t amp_t sum_i sum_c g_{t,i}(c) beta_{i,c}[a_i(e)] prod_{m != i}
// P1[t][m][a_m(e)], plus for the constant c0 the same with the factors of
// 1 (projection e_0, value 1 at both faces): the load of boundary data that
// is the restriction of a separable sum.
__global__ void dirichlet_load_kernel(long long dof, int d, int kp1, int H, long long ntuples,
                                      const int* __restrict__ levels, const long long* __restrict__ offsets,
                                      int nterms, const double* __restrict__ amp, const double* __restrict__ P1,
                                      const double* __restrict__ gface, const double* __restrict__ beta, double c0,
                                      double* __restrict__ b) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < dof;
         e += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = ntuples;  // offsets[lo] <= e < offsets[hi]
        while (hi - lo > 1) {
            const long long mid = (lo + hi) / 2;
            if (offsets[mid] <= e) lo = mid;
            else hi = mid;
        }
        long long loc = e - offsets[lo];
        int a[SGK_MAX_DIM];
        for (int m = d - 1; m >= 0; --m) {
            const int l = levels[lo * d + m];
            const int nl = l == 0 ? kp1 : kp1 << (l - 1);
            const int t = (int)(loc % nl);
            loc /= nl;
            a[m] = (l == 0 ? 0 : kp1 << (l - 1)) + t;
        }
        double acc = 0.0;
        for (int i = 0; i < d; ++i) {
            const double b0 = beta[((long long)i * 2 + 0) * H + a[i]], b1 = beta[((long long)i * 2 + 1) * H + a[i]];
            for (int t = 0; t < nterms; ++t) {
                const double gf = gface[t * d + i];
                if (gf == 0.0) continue;
                double prod = amp[t] * gf * (b0 + b1);
                for (int m = 0; m < d; ++m)
                    if (m != i) prod *= P1[((long long)t * d + m) * H + a[m]];
                acc += prod;
            }
            if (c0 != 0.0) {
                bool rest0 = true;
                for (int m = 0; m < d; ++m)
                    if (m != i && a[m] != 0) rest0 = false;
                if (rest0) acc += c0 * (b0 + b1);
            }
        }
        b[e] = acc;
    }
}

}  // namespace

// ------------------------------------------------------------ host side ---

int reaction_degree(const ReactionDev& rx) {
    int p = 0;
    for (int m = 0; m < rx.nmono; ++m) {
        int s = 0;
        for (int r = 0; r < rx.nspecies; ++r) s += rx.exps[m][r];
        p = std::max(p, s);
    }
    return p;
}

void quad_build(Quad& Q, const sgk_index* idx, int q, int nspecies, bool need_jacobian) {
    sgk_ctx* ctx = idx->ctx;
    const int d = idx->d, N = idx->n, k = idx->k, kp1 = k + 1;
    Q.d = d;
    Q.N = N;
    Q.kp1 = kp1;
    Q.q = q;
    Q.nspecies = nspecies;
    Q.H = kp1 << N;
    Q.idx = idx;
    build_transform_tables(N, k, Q.tab);
    Q.tab.T.upload(ctx->stream);
    Q.tab.Tt.upload(ctx->stream);
    // R_i layouts: blocks over tuples of directions i..d-1, each H^i x prod n
    const int H = Q.H;
    Q.layout_offsets.assign(d + 1, {});
    Q.layout_size.assign(d + 1, 0);
    for (int i = 0; i <= d; ++i) {
        auto tl = tuples_lex(d - i, N);
        std::vector<long long> off(tl.size() + 1, 0);
        long long Hi = 1;
        for (int m = 0; m < i; ++m) Hi *= H;
        for (size_t t = 0; t < tl.size(); ++t) {
            long long sz = Hi;
            for (int v : tl[t]) sz *= level_count(v, kp1);
            off[t + 1] = off[t] + sz;
        }
        Q.layout_offsets[i] = off;
        Q.layout_size[i] = off.back();
    }
    SGK_REQUIRE(Q.layout_size[0] == idx->dof, SGK_EINVAL, "internal layout mismatch");
    // fiber plans for direction i: groups over tuples of directions i+1..d-1
    for (int i = 0; i < d; ++i) {
        std::vector<FiberGroup> groups;
        auto gl = tuples_lex(d - i - 1, N);
        long long O = 1;
        for (int m = 0; m < i; ++m) O *= H;
        SGK_REQUIRE(O < (1LL << 31), SGK_EUNSUPPORTED, "full grid too large for the transform plan");
        for (size_t gi = 0; gi < gl.size(); ++gi) {
            const auto& g = gl[gi];
            FiberGroup fg{};
            int rest = 0;
            long long I = 1;
            for (int v : g) {
                rest += v;
                I *= level_count(v, kp1);
            }
            fg.nlev = N - rest + 1;
            fg.O = (int)O;
            fg.I = (int)I;
            std::vector<int> t(g.size() + 1);
            for (int l = 0; l < fg.nlev; ++l) {
                t[0] = l;
                for (size_t j = 0; j < g.size(); ++j) t[j + 1] = g[j];
                fg.cbase[l] = Q.layout_offsets[i][tuple_rank(t, N)];
            }
            fg.fbase = Q.layout_offsets[i + 1][gi];
            groups.push_back(fg);
        }
        const long long ri = Q.layout_size[i], ro = Q.layout_size[i + 1];
        finalize_plan(Q.fwd[i][0], groups, kp1, H, FIBER_FWD, sizeof(double), 40 * 1024, ri, ro, ctx->stream);
        finalize_plan(Q.fwd[i][1], groups, kp1, H, FIBER_FWD, sizeof(float), 40 * 1024, ri, ro, ctx->stream);
        finalize_plan(Q.bwd[i][0], groups, kp1, H, FIBER_BWD, sizeof(double), 40 * 1024, ro, ri, ctx->stream);
        finalize_plan(Q.bwd[i][1], groups, kp1, H, FIBER_BWD, sizeof(float), 40 * 1024, ro, ri, ctx->stream);
    }
    // Gauss tables: B[g][r] = h^{-1/2} sqrt(2r+1) P_r(xi_g); w1[g] = h w_g / 2
    std::vector<double> xg, wg;
    gauss_legendre(q, xg, wg);
    const double h = std::ldexp(1.0, -N);
    std::vector<double> B(q * kp1), w1(q);
    for (int g = 0; g < q; ++g) {
        std::vector<double> P(kp1 + 1, 0.0);
        P[0] = 1.0;
        P[1] = xg[g];
        for (int r = 1; r < kp1; ++r) P[r + 1] = ((2 * r + 1) * xg[g] * P[r] - r * P[r - 1]) / (r + 1);
        for (int r = 0; r < kp1; ++r) B[g * kp1 + r] = std::sqrt(2.0 * r + 1.0) * P[r] / std::sqrt(h);
        w1[g] = 0.5 * h * wg[g];
    }
    Q.B_host = B;
    Q.w_host = w1;
    Q.B64.upload(B, ctx->stream);
    Q.w64.upload(w1, ctx->stream);
    std::vector<float> Bf(B.begin(), B.end()), wf(w1.begin(), w1.end());
    Q.B32.alloc(Bf.size());
    Q.B32.upload(Bf.data(), Bf.size(), ctx->stream);
    Q.w32.alloc(wf.size());
    Q.w32.upload(wf.data(), wf.size(), ctx->stream);
    SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    Q.full_size = Q.layout_size[d];
    Q.maxstage = ipow(std::max(kp1, q), d);
    (void)need_jacobian;
}

template <typename T>
static const T* tvals(const Csr& c) {
    return sizeof(T) == 8 ? reinterpret_cast<const T*>(c.d_val.p) : reinterpret_cast<const T*>(c.d_valf.p);
}

template <typename T>
void quad_forward(sgk_ctx* ctx, const Quad& Q, const T* in, T* final_nodal, T* tmp, int ndims) {
    const int prec = sizeof(T) == 8 ? 0 : 1;
    const T* src = in;
    for (int i = 0; i < ndims; ++i) {
        T* dst = ((ndims - 1 - i) % 2 == 0) ? final_nodal : tmp;
        launch_pyr<T>(ctx, Q.fwd[i][prec], FIBER_FWD, src, dst, Q.H, Q.kp1, Q.tab.two_scale.data());
        src = dst;
    }
}

template <typename T>
void quad_backward(sgk_ctx* ctx, const Quad& Q, T* moments, T* tmp, T* out, int ndims) {
    const int prec = sizeof(T) == 8 ? 0 : 1;
    const T* src = moments;
    for (int i = ndims - 1; i >= 0; --i) {
        T* dst = i == 0 ? out : (((ndims - 1 - i) % 2 == 0) ? tmp : moments);
        launch_pyr<T>(ctx, Q.bwd[i][prec], FIBER_BWD, src, dst, Q.H, Q.kp1, Q.tab.two_scale.data());
        src = dst;
    }
}

template <typename T>
void quad_cells(sgk_ctx* ctx, const Quad& Q, const ReactionDev& rx, bool jac, const T* const* u, const T* const* w,
                T* const* out) {
    CellParams<T> p{};
    p.d = Q.d;
    p.kp1 = Q.kp1;
    p.q = Q.q;
    p.ncell1 = 1 << Q.N;
    p.H = Q.H;
    p.maxstage = Q.maxstage;
    p.nspecies = Q.nspecies;
    p.ncells = 1;
    for (int m = 0; m < Q.d; ++m) p.ncells *= p.ncell1;
    long long hp = 1;
    for (int m = 0; m < Q.d; ++m) {
        p.Hpow[m] = hp;
        hp *= Q.H;
    }
    for (int s = 0; s < Q.nspecies; ++s) {
        p.u[s] = u[s];
        p.w[s] = jac ? w[s] : nullptr;
        p.out[s] = out[s];
    }
    p.B = sizeof(T) == 8 ? reinterpret_cast<const T*>(Q.B64.p) : reinterpret_cast<const T*>(Q.B32.p);
    p.w1 = sizeof(T) == 8 ? reinterpret_cast<const T*>(Q.w64.p) : reinterpret_cast<const T*>(Q.w32.p);
    p.rx = rx;
    const int nsets = jac ? 2 * Q.nspecies : Q.nspecies;
    const size_t per_cell = (size_t)nsets * 2 * Q.maxstage * sizeof(T);
    const size_t budget = 96 * 1024;
    p.cpb = (int)std::max<size_t>(1, std::min<size_t>(64, budget / per_cell));
    const size_t smem = per_cell * p.cpb;
    SGK_REQUIRE(smem <= ctx->smem_optin, SGK_EUNSUPPORTED, "cell quadrature tile exceeds shared memory");
    long long blocks = (p.ncells + p.cpb - 1) / p.cpb;
    const int grid = (int)std::min<long long>(blocks, (long long)ctx->num_sms * 4);
    KTimer kt(ctx, KC_CELL);
    if (jac) {
        allow_max_dynamic_smem(ctx->smem_optin, cell_kernel<T, 1>);
        cell_kernel<T, 1><<<grid, 256, smem, ctx->stream>>>(p);
    } else {
        allow_max_dynamic_smem(ctx->smem_optin, cell_kernel<T, 0>);
        cell_kernel<T, 0><<<grid, 256, smem, ctx->stream>>>(p);
    }
    check_launch("cell_kernel");
    count_launch(ctx);
}

template void quad_forward<double>(sgk_ctx*, const Quad&, const double*, double*, double*, int);
template void quad_forward<float>(sgk_ctx*, const Quad&, const float*, float*, float*, int);
template void quad_backward<double>(sgk_ctx*, const Quad&, double*, double*, double*, int);
template void quad_backward<float>(sgk_ctx*, const Quad&, float*, float*, float*, int);
template void quad_forward<dfloat>(sgk_ctx*, const Quad&, const dfloat*, dfloat*, dfloat*, int);
template void quad_backward<dfloat>(sgk_ctx*, const Quad&, dfloat*, dfloat*, dfloat*, int);
template void quad_cells<double>(sgk_ctx*, const Quad&, const ReactionDev&, bool, const double* const*,
                                 const double* const*, double* const*);
template void quad_cells<float>(sgk_ctx*, const Quad&, const ReactionDev&, bool, const float* const*,
                                const float* const*, float* const*);

// P1[(t d + m) H + a] = int g_{t,m}(2 pi w_{t,m} x) v_a(x) dx, the 1D
// projections of the factors of a separable sum (12-point Gauss per finest
// cell, then the transposed change of basis); damp receives amp.
static void separable_factors_dev(sgk_ctx* ctx, const sgk_index* idx, const Tables1D& tab, int nterms,
                                  const double* amp, const int* wavenum, const int* kind, DevBuf<double>& damp,
                                  DevBuf<double>& P1) {
    const int d = idx->d, N = idx->n, kp1 = idx->k + 1, H = kp1 << N;
    if (nterms <= 0) return;
    std::vector<double> xg, wg;
    gauss_legendre(12, xg, wg);
    DevBuf<double> dx, dw, fine;
    DevBuf<int> dwn, dkind;
    dx.upload(xg, ctx->stream);
    dw.upload(wg, ctx->stream);
    const long long nvec = (long long)nterms * d;
    std::vector<int> wn(wavenum, wavenum + (size_t)nterms * d), kd(kind, kind + (size_t)nterms * d);
    std::vector<double> am(amp, amp + nterms);
    dwn.upload(wn, ctx->stream);
    dkind.upload(kd, ctx->stream);
    damp.upload(am, ctx->stream);
    fine.alloc(nvec * H);
    P1.alloc(nvec * H);
    const int grid = (int)std::min<long long>((nvec * H + 255) / 256, ctx->num_sms * 8LL);
    proj_fine_kernel<<<grid, 256, 0, ctx->stream>>>(nterms, d, N, kp1, dwn.p, dkind.p, dx.p, dw.p, 12, fine.p);
    check_launch("proj_fine_kernel");
    proj_hier_kernel<<<grid, 256, 0, ctx->stream>>>(nvec, H, tab.Tt.d_ptr.p, tab.Tt.d_col.p, tab.Tt.d_val.p,
                                                     fine.p, P1.p);
    check_launch("proj_hier_kernel");
    count_launch(ctx, 2);
    SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));  // host vectors above go out of scope
}

void project_separable_dev(sgk_ctx* ctx, const sgk_index* idx, const Tables1D& tab, int nterms, const double* amp,
                           const int* wavenum, const int* kind, double c0, double* U) {
    const int d = idx->d, N = idx->n, kp1 = idx->k + 1, H = kp1 << N;
    DevBuf<double> damp, P1;
    separable_factors_dev(ctx, idx, tab, nterms, amp, wavenum, kind, damp, P1);
    const int grid = (int)std::min<long long>((idx->dof + 255) / 256, ctx->num_sms * 8LL);
    proj_product_kernel<<<grid, 256, 0, ctx->stream>>>(idx->dof, d, kp1, H, idx->ntuples, idx->d_levels.p,
                                                        reinterpret_cast<const long long*>(idx->d_offsets.p), nterms,
                                                        damp.p, P1.p, c0, U);
    check_launch("proj_product_kernel");
    count_launch(ctx);
    SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    (void)N;
}

void dirichlet_load_dev(sgk_ctx* ctx, const sgk_index* idx, const Tables1D& tab, const double* kappa, double sigma,
                        int nterms, const double* amp, const int* wavenum, const int* kind, double c0, double* b) {
    const int d = idx->d, N = idx->n, kp1 = idx->k + 1, H = kp1 << N;
    const double h = std::ldexp(1.0, -N);
    // one-sided traces v(0+), v'(0+), v(1-), v'(1-) of every 1D hierarchical
    // function from its Legendre coefficients on the first and last finest
    // cells (phi_p = h^{-1/2} sqrt(2p+1) P_p(2(x - x_c)/h - 1):
    // P_p(-1) = (-1)^p, P_p'(-1) = (-1)^{p+1} p(p+1)/2, P_p(1) = 1,
    // P_p'(1) = p(p+1)/2)
    std::vector<double> v0(H, 0.0), d0(H, 0.0), v1(H, 0.0), d1(H, 0.0);
    const double rh = 1.0 / std::sqrt(h);
    for (int a = 0; a < H; ++a)
        for (int e = tab.Tt.ptr[a]; e < tab.Tt.ptr[a + 1]; ++e) {
            const int y = tab.Tt.col[e], p = y % kp1;
            const double t = tab.Tt.val[e], nrm = rh * std::sqrt(2.0 * p + 1.0), dp = 0.5 * p * (p + 1);
            const double sgn = (p % 2) ? -1.0 : 1.0;
            if (y < kp1) {
                v0[a] += t * nrm * sgn;
                d0[a] += t * nrm * (-sgn) * dp * 2.0 / h;
            }
            if (y >= H - kp1) {
                v1[a] += t * nrm;
                d1[a] += t * nrm * dp * 2.0 / h;
            }
        }
    // per direction i and face c (outward normal -1 at 0, +1 at 1):
    // beta = -kappa_i (n v' - sigma/h v), the face factor of the load
    std::vector<double> beta((size_t)d * 2 * H);
    for (int i = 0; i < d; ++i)
        for (int a = 0; a < H; ++a) {
            beta[((size_t)i * 2 + 0) * H + a] = -kappa[i] * (-d0[a] - sigma / h * v0[a]);
            beta[((size_t)i * 2 + 1) * H + a] = -kappa[i] * (d1[a] - sigma / h * v1[a]);
        }
    // the data's factors at the faces: sin(2 pi w c) = 0, cos(2 pi w c) = 1
    // for integer w and c in {0, 1}
    std::vector<double> gface((size_t)std::max(nterms, 1) * d, 0.0);
    for (int t = 0; t < nterms * d; ++t) gface[t] = kind[t] == 1 ? 1.0 : 0.0;
    DevBuf<double> damp, P1, dbeta, dgf;
    separable_factors_dev(ctx, idx, tab, nterms, amp, wavenum, kind, damp, P1);
    dbeta.upload(beta, ctx->stream);
    dgf.upload(gface, ctx->stream);
    const int grid = (int)std::min<long long>((idx->dof + 255) / 256, ctx->num_sms * 8LL);
    dirichlet_load_kernel<<<grid, 256, 0, ctx->stream>>>(idx->dof, d, kp1, H, idx->ntuples, idx->d_levels.p,
                                                          reinterpret_cast<const long long*>(idx->d_offsets.p),
                                                          nterms, damp.p, P1.p, dgf.p, dbeta.p, c0, b);
    check_launch("dirichlet_load_kernel");
    count_launch(ctx);
    SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
}
