// Rys quadrature nodes and weights on the device (tables written by gen_rys.py).
//
// For the Boys weight exp(-T t^2) on t in [0, 1], the n-point rule
//   integral_0^1 f(t^2) exp(-T t^2) dt = sum_i w_i f(u_i)
// is exact for polynomials f of degree < 2n; an electron-repulsion integral of
// total angular momentum L is such a polynomial with n = L / 2 + 1 (Rys,
// Dupuis and King, J. Comput. Chem. 4, 154 (1983)).  Below rys_switch(n) the
// nodes and weights are degree-11 polynomials on unit intervals of T; from
// there on their large-T limit u_i = x_i^2 / T, w_i = W_i / sqrt(T) (x_i, W_i:
// the positive Gauss-Hermite nodes and weights of order 2n).
#pragma once
#include "rys_tables.h"

namespace hf {

template <int n>
__device__ __forceinline__ const double* rys_table();
template <>
__device__ __forceinline__ const double* rys_table<1>() { return kRysTab1; }
template <>
__device__ __forceinline__ const double* rys_table<2>() { return kRysTab2; }
template <>
__device__ __forceinline__ const double* rys_table<3>() { return kRysTab3; }
template <>
__device__ __forceinline__ const double* rys_table<4>() { return kRysTab4; }
template <>
__device__ __forceinline__ const double* rys_table<5>() { return kRysTab5; }

template <int n>
__device__ __forceinline__ const double* rys_herm_x();
template <>
__device__ __forceinline__ const double* rys_herm_x<1>() { return kRysHermX1; }
template <>
__device__ __forceinline__ const double* rys_herm_x<2>() { return kRysHermX2; }
template <>
__device__ __forceinline__ const double* rys_herm_x<3>() { return kRysHermX3; }
template <>
__device__ __forceinline__ const double* rys_herm_x<4>() { return kRysHermX4; }
template <>
__device__ __forceinline__ const double* rys_herm_x<5>() { return kRysHermX5; }

template <int n>
__device__ __forceinline__ const double* rys_herm_w();
template <>
__device__ __forceinline__ const double* rys_herm_w<1>() { return kRysHermW1; }
template <>
__device__ __forceinline__ const double* rys_herm_w<2>() { return kRysHermW2; }
template <>
__device__ __forceinline__ const double* rys_herm_w<3>() { return kRysHermW3; }
template <>
__device__ __forceinline__ const double* rys_herm_w<4>() { return kRysHermW4; }
template <>
__device__ __forceinline__ const double* rys_herm_w<5>() { return kRysHermW5; }

// u[n] nodes (t^2) and w[n] weights of the n-point rule at T >= 0.
template <int n>
__device__ __forceinline__ void rys_rule(double T, double* u, double* w)
{
    if (T < (double)rys_switch(n)) {
        const int k = (int)T;
        const double x = 2.0 * (T - (double)k) - 1.0;
        const double* __restrict__ c = rys_table<n>() + (size_t)k * (2 * n) * (kRysDeg + 1);
#pragma unroll
        for (int i = 0; i < 2 * n; i++) {
            const double* ci = c + i * (kRysDeg + 1);
            double v = ci[kRysDeg];
#pragma unroll
            for (int j = kRysDeg - 1; j >= 0; j--) v = fma(v, x, ci[j]);
            if (i < n)
                u[i] = v;
            else
                w[i - n] = v;
        }
    } else {
        const double rs = rsqrt(T);
        const double rT = rs * rs;
        const double* hx = rys_herm_x<n>();
        const double* hw = rys_herm_w<n>();
#pragma unroll
        for (int i = 0; i < n; i++) {
            u[i] = hx[i] * rT;
            w[i] = hw[i] * rs;
        }
    }
}

}  // namespace hf
