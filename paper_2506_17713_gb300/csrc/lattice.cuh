// Velocity sets and MRT moment bases of the CUDA path (compile-time constants).
//
// D2Q9 and D3Q19 of Section 2.1 (Eq. lbe). The MRT bases are the Gram-Schmidt
// polynomial bases cited there for MRT (Lallemand & Luo 2000 / McCracken &
// Abraham 2005 for D2Q9, d'Humieres et al. 2002 for D3Q19); every entry is
// evaluated at compile time from the moment polynomial, so unrolled loops over
// (moment, direction) fold to straight-line adds of +-populations.
#pragma once

#include <cstdint>

namespace lbm {

struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int D = 2;
    // 0: rest, 1-4: axis links, 5-8: diagonals
    __host__ __device__ static constexpr int ex(int i)
    {
        constexpr int v[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        return v[i];
    }
    __host__ __device__ static constexpr int ey(int i)
    {
        constexpr int v[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        return v[i];
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i)
    {
        constexpr int v[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        return v[i];
    }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    // moment polynomial a of velocity i (rho, e, eps, jx, qx, jy, qy, pxx, pxy)
    __host__ __device__ static constexpr int M(int a, int i)
    {
        const int x = ex(i), y = ey(i), c2 = x * x + y * y;
        switch (a) {
        case 0: return 1;
        case 1: return 3 * c2 - 4;
        case 2: return (9 * c2 * c2 - 21 * c2 + 8) / 2;
        case 3: return x;
        case 4: return (3 * c2 - 5) * x;
        case 5: return y;
        case 6: return (3 * c2 - 5) * y;
        case 7: return x * x - y * y;
        case 8: return x * y;
        }
        return 0;
    }
    __host__ __device__ static constexpr bool conserved(int a) { return a == 0 || a == 3 || a == 5; }
    __host__ __device__ static constexpr bool stress(int a) { return a == 7 || a == 8; }
};

struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int D = 3;
    // 0: rest, 1-6: axis links (+x,-x,+y,-y,+z,-z), 7-18: edge links in opposite pairs
    __host__ __device__ static constexpr int ex(int i)
    {
        constexpr int v[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return v[i];
    }
    __host__ __device__ static constexpr int ey(int i)
    {
        constexpr int v[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return v[i];
    }
    __host__ __device__ static constexpr int ez(int i)
    {
        constexpr int v[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return v[i];
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i % 2 ? i + 1 : i - 1); }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    // moment polynomial a of velocity i, d'Humieres et al. (2002) order
    __host__ __device__ static constexpr int M(int a, int i)
    {
        const int x = ex(i), y = ey(i), z = ez(i), c2 = x * x + y * y + z * z;
        switch (a) {
        case 0: return 1;
        case 1: return 19 * c2 - 30;
        case 2: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
        case 3: return x;
        case 4: return (5 * c2 - 9) * x;
        case 5: return y;
        case 6: return (5 * c2 - 9) * y;
        case 7: return z;
        case 8: return (5 * c2 - 9) * z;
        case 9: return 3 * x * x - c2;
        case 10: return (3 * c2 - 5) * (3 * x * x - c2);
        case 11: return y * y - z * z;
        case 12: return (3 * c2 - 5) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return (y * y - z * z) * x;
        case 17: return (z * z - x * x) * y;
        case 18: return (x * x - y * y) * z;
        }
        return 0;
    }
    __host__ __device__ static constexpr bool conserved(int a) { return a == 0 || a == 3 || a == 5 || a == 7; }
    __host__ __device__ static constexpr bool stress(int a)
    {
        return a == 9 || a == 11 || a == 13 || a == 14 || a == 15;
    }
};

// squared norm of moment row a (the basis is orthogonal, so M^-1 = M^T diag(1/norm))
template <class L>
__host__ __device__ constexpr int mrt_norm(int a)
{
    int s = 0;
    for (int i = 0; i < L::Q; ++i) s += L::M(a, i) * L::M(a, i);
    return s;
}

}  // namespace lbm
