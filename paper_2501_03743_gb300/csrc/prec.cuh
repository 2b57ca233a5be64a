// Chebyshev polynomial preconditioner: z = p(D^-1 A) D^-1 v, the result of
// `degree` steps of Chebyshev acceleration (Saad, Iterative Methods for
// Sparse Linear Systems, Sec. 12.3) on D^-1 A y = D^-1 v from y = 0 over the
// interval [lmin, lmax] of D^-1 A.  With theta = (lmax+lmin)/2,
// delta = (lmax-lmin)/2, sigma = theta/delta:
//   g = D^-1 v, rho_0 = 1/sigma, d_0 = g/theta, z = d_0, res = g
//   k = 1..degree-1: res -= D^-1 A d_{k-1}; rho_k = 1/(2 sigma - rho_{k-1});
//                    d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k/delta) res; z += d_k
// so 1 - lambda p(lambda) = T_degree((theta - lambda)/delta) / T_degree(sigma).
// One apply costs degree-1 SpMVs; each step is one fused kernel.
#pragma once

#include <vector>

#include "common.cuh"
#include "spmv.cuh"

namespace sscg {

namespace {

template <class A>
__global__ void __launch_bounds__(kThreads) k_cheb_first(int n, const typename A::S* __restrict__ v,
                                                         const typename A::S* __restrict__ dinv,
                                                         typename A::S* __restrict__ z, typename A::S* __restrict__ res,
                                                         typename A::S* __restrict__ d, double inv_theta,
                                                         const Ctrl* ctrl) {
    using R = typename A::R;
    if (ctrl && __ldcg(&ctrl->done)) return;
    const R it = A::from_d(inv_theta);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        R g = A::mul(A::ld(dinv + i), A::ld(v + i));
        R d0 = A::mul(g, it);
        A::st(z + i, d0);
        if (res) {
            A::st(res + i, g);
            A::st(d + i, d0);
        }
    }
}

template <class A, int VM>
__global__ void __launch_bounds__(kThreads) k_cheb_step(MatView M, const typename A::S* __restrict__ dinv,
                                                        const typename A::S* __restrict__ d_in,
                                                        typename A::S* __restrict__ d_out,
                                                        typename A::S* __restrict__ res, typename A::S* __restrict__ z,
                                                        double c1, double c2, const Ctrl* ctrl) {
    using R = typename A::R;
    if (ctrl && __ldcg(&ctrl->done)) return;
    extern __shared__ __align__(16) char smem_raw[];
    char* smem = align128(smem_raw);
    const R C1 = A::from_d(c1), C2 = A::from_d(c2);
    spmv_pipe<A, VM, kStages>(
        M, smem, [&](int c) { return A::ldg(d_in + c); },
        [&](int row, R q) {
            R rs = A::sub(A::ld(res + row), A::mul(A::ld(dinv + row), q));
            R dn = A::fma(C1, A::ldg(d_in + row), A::mul(C2, rs));
            A::st(res + row, rs);
            A::st(d_out + row, dn);
            A::st(z + row, A::add(A::ld(z + row), dn));
        },
        const_cast<Ctrl*>(ctrl));
}

// Host side: launch the kernels of one apply z = B^-1 v on `st`.
// tmp holds 3 vectors of ldn elements (res, d0, d1).
template <class A, int VM>
struct ChebPrec {
    using S = typename A::S;
    int degree;
    double theta, delta;
    std::vector<double> c1, c2;
    ChebPrec(int deg, double lmin, double lmax) : degree(deg) {
        theta = 0.5 * (lmax + lmin);
        delta = 0.5 * (lmax - lmin);
        double sigma = theta / delta, rho = 1.0 / sigma;
        for (int k = 1; k < deg; k++) {
            double rn = 1.0 / (2.0 * sigma - rho);
            c1.push_back(rn * rho);
            c2.push_back(2.0 * rn / delta);
            rho = rn;
        }
    }
    // Returns the number of kernels launched.
    int apply(const MatView& M, const S* dinv, const S* v, S* z, S* tmp, size_t ldn, int G, int Gs, size_t smem,
              cudaStream_t st, const Ctrl* ctrl) const {
        S* res = tmp;
        S* d[2] = {tmp + ldn, tmp + 2 * ldn};
        k_cheb_first<A><<<G, kThreads, 0, st>>>(M.n, v, dinv, z, degree > 1 ? res : nullptr, d[0], 1.0 / theta,
                                                ctrl);
        for (int k = 1; k < degree; k++)
            k_cheb_step<A, VM><<<Gs, kThreads, smem, st>>>(M, dinv, d[(k - 1) & 1], d[k & 1], res, z, c1[k - 1],
                                                           c2[k - 1], ctrl);
        return degree;
    }
};

}  // namespace

}  // namespace sscg
