// CUDA kernels of the Shan-Chen multiphase lattice Boltzmann step (sm_103a).
//
// Data layout in HBM: populations are structure-of-arrays, f[k][i][z][y][x]
// (x fastest), so a warp touching 32 consecutive x of one direction plane
// reads or writes 128 contiguous bytes (FP32). Two population buffers are
// kept: the step PULLS post-collision values f*_i(x - e_i) from one buffer
// (streaming, Eq. lbe_steps) and writes the new post-collision values to the
// other, at the node itself (aligned, coalesced stores).
//
// A step is two passes over the lattice:
//   density pass : gather -> rho^k -> psi^k (and U^k) (Eqs. macroeq_mcp, eos_potential)
//   [virtual pass: rho_s, psi_s at boundary solids (Eq. improved_virtual_density)]
//   collide pass : gather -> rho, j -> force from the psi/U stencil
//                  (Eq. software_ff_force_mcmp) -> BGK/MRT (Eq. collision_model)
//                  -> EDM (Eq. edm) -> store
// The density and collide passes sum the same gathered values in the same
// order, so both see bit-identical rho.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <utility>

#include "args.h"
#include "lattice.cuh"

// Per-node arithmetic is __host__ __device__ so that host-side harnesses can
// exercise exactly the arithmetic of the kernels.
#define LBM_HD __host__ __device__ __forceinline__

namespace lbm {

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1, so that
// table lookups inside the body are constant expressions (bound to constexpr
// locals) rather than calls the optimiser may or may not fold.
template <class F, int... I>
LBM_HD void static_for_impl(F&& f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
LBM_HD void static_for(F&& f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// first member i (i < opp(i)) of the p-th opposite pair of the velocity set
template <class L>
LBM_HD constexpr int pair_first(int p)
{
    int n = 0;
    for (int i = 1; i < L::Q; ++i)
        if (i < L::opp(i)) {
            if (n == p) return i;
            ++n;
        }
    return -1;
}

// moment a of the MRT basis is even under e -> -e (sees pair sums only)
template <class L>
LBM_HD constexpr bool mrt_even(int a)
{
    for (int i = 1; i < L::Q; ++i)
        if (L::M(a, i) != L::M(a, L::opp(i))) return false;
    return true;
}

// Double-float ("float-float") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2.
// Error-free transformations (Knuth's TwoSum, FMA-based TwoProd) give about 44
// significant bits from FP32 operations. Used where FP32 rounding would be
// amplified by the interface dynamics (interaction force, EOS). For T = double
// the same interface degrades to plain double arithmetic.
template <typename T>
struct FF {
    T hi, lo;
};
template <typename T>
LBM_HD FF<T> ff_two_sum(T a, T b)
{
    const T s = a + b;
    const T bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
template <typename T>
LBM_HD FF<T> ff_two_prod(T a, T b)
{
    const T p = a * b;
    return {p, fma(a, b, -p)};
}
template <typename T>
LBM_HD FF<T> ff_add(FF<T> a, FF<T> b)
{
    FF<T> s = ff_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return ff_two_sum(s.hi, s.lo);
}
template <typename T>
LBM_HD FF<T> ff_mul(FF<T> a, FF<T> b)
{
    FF<T> p = ff_two_prod(a.hi, b.hi);
    p.lo = fma(a.hi, b.lo, fma(a.lo, b.hi, p.lo));
    return ff_two_sum(p.hi, p.lo);
}
template <typename T>
LBM_HD FF<T> ff_mul(FF<T> a, T b)
{
    FF<T> p = ff_two_prod(a.hi, b);
    p.lo = fma(a.lo, b, p.lo);
    return ff_two_sum(p.hi, p.lo);
}
template <typename T>
LBM_HD FF<T> ff_div(FF<T> a, FF<T> b)
{
    const T q1 = a.hi / b.hi;
    const FF<T> r = ff_add(a, ff_mul(b, -q1));
    const T q2 = r.hi / b.hi;
    return ff_two_sum(q1, q2);
}
template <typename T>
LBM_HD FF<T> ff_of(T a) { return {a, T(0)}; }

// correctly rounded reciprocal (one short hardware sequence instead of a division)
LBM_HD float rcp(float x)
{
#ifdef __CUDA_ARCH__
    return __frcp_rn(x);
#else
    return 1.0f / x;
#endif
}
LBM_HD double rcp(double x)
{
#ifdef __CUDA_ARCH__
    return __drcp_rn(x);
#else
    return 1.0 / x;
#endif
}

// Compensated summation (Neumaier's variant of Kahan summation): the running
// sum carries the rounding error of every addition in a second register, so
// rho = sum_i f_i and j = sum_i f_i e_i come out within about one rounding of
// the exact sums of the stored values.
template <typename T>
struct CSum {
    T s = T(0), c = T(0);
    LBM_HD void add(T v)
    {
        const T t = s + v;
        c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
    LBM_HD T value() const { return s + c; }
};

// Moment-space form of the EDM shift: for the second-order equilibrium,
//   m_a^eq(rho, u') - m_a^eq(rho, u) = rho [3 sum_d A_ad du_d + sum_{d<=d'} B_add' dq_dd'],
//   dq_dd' = u'_d u'_d' - u_d u_d', with constants of the basis
//   A_ad = sum_i M_ai w_i e_id,  B_add' = (2 - [d=d']) (4.5 sum_i M_ai w_i e_id e_id' - 1.5 [d=d'] sum_i M_ai w_i).
template <class L>
LBM_HD constexpr int e_of(int i, int d)
{
    return d == 0 ? L::ex(i) : (d == 1 ? L::ey(i) : L::ez(i));
}
template <class L>
LBM_HD constexpr double edm_A(int a, int d)
{
    double s = 0.0;
    for (int i = 0; i < L::Q; ++i) s += L::M(a, i) * L::w(i) * e_of<L>(i, d);
    return s;
}
template <class L>
LBM_HD constexpr double edm_B(int a, int d, int dp)
{
    double s2 = 0.0, s0 = 0.0;
    for (int i = 0; i < L::Q; ++i) {
        s2 += L::M(a, i) * L::w(i) * e_of<L>(i, d) * e_of<L>(i, dp);
        s0 += L::M(a, i) * L::w(i);
    }
    const double b = 4.5 * s2 - (d == dp ? 1.5 * s0 : 0.0);
    return d == dp ? b : 2.0 * b;
}

// ---------------------------------------------------------------------------
// Equation of state and pseudopotential (Section 2.2, Eq. eos_potential)
// ---------------------------------------------------------------------------

template <typename T>
LBM_HD T eos_pressure(const Params<T>& P, int k, T rho)
{
    const T a = P.eos_a[k], b = P.eos_b[k], RT = P.RT[k];
    switch (P.eos[k]) {
    case EOS_CS: {
        const T eta = b * rho * T(0.25);
        const T om = T(1) - eta;
        return rho * RT * (T(1) + eta * (T(1) + eta * (T(1) - eta))) / (om * om * om) - a * rho * rho;
    }
    case EOS_PR:
        return rho * RT / (T(1) - b * rho)
               - a * P.alphaT[k] * rho * rho / (T(1) + b * rho * (T(2) - b * rho));
    case EOS_VDW:
        return rho * RT / (T(1) - b * rho) - a * rho * rho;
    case EOS_RK:
        return rho * RT / (T(1) - b * rho) - a * rho * rho / (P.sqrtT[k] * (T(1) + b * rho));
    default:  // EOS_RKS
        return rho * RT / (T(1) - b * rho) - a * P.alphaT[k] * rho * rho / (T(1) + b * rho);
    }
}

// FP32 pseudopotential energy in double-float arithmetic. Every EOS here can be
// written p = rho N(rho) / D(rho) with a polynomial numerator N (degree 2, or 4
// for Carnahan-Starling) and a cancellation-free denominator D (powers of 1 - b rho,
// 1 + b rho, 1 + 2 b rho - b^2 rho^2); the host folds R T, a, b and alpha(T) into
// the coefficients of N. In a stiff liquid the terms of N nearly cancel, so N is
// evaluated as hi + lo (Horner), D in plain FP32 with fused multiply-adds, and
//   U = alpha p - c_s^2 rho = rho (alpha N / D - 1/3)
// as hi + lo.
template <typename T>
LBM_HD T eos_denominator(const Params<T>& P, int k, T rho)
{
    const T b = P.eos_b[k];
    switch (P.eos[k]) {
    case EOS_CS: {
        const T om = fma(T(-0.25) * b, rho, T(1));
        return om * om * om;
    }
    case EOS_PR: {
        const T br = b * rho;
        return fma(-b, rho, T(1)) * fma(br, T(2) - br, T(1));
    }
    case EOS_VDW: return fma(-b, rho, T(1));
    default: return fma(-b * b, rho * rho, T(1));  // RK, RKS: (1 - b rho)(1 + b rho)
    }
}

template <int DEG, typename T>
LBM_HD FF<T> eos_numerator(const Params<T>& P, int k, T rho)
{
    FF<T> n = {P.eos_c[k][DEG], P.eos_c_lo[k][DEG]};
#pragma unroll
    for (int d = DEG - 1; d >= 0; --d) n = ff_add(ff_mul(n, rho), FF<T>{P.eos_c[k][d], P.eos_c_lo[k][d]});
    return n;
}

template <typename T>
LBM_HD FF<T> eos_energy_ff(const Params<T>& P, int k, T rho)
{
    const FF<T> n = P.eos[k] == EOS_CS ? eos_numerator<4>(P, k, rho) : eos_numerator<2>(P, k, rho);
    // alpha N / D: the quotient of hi + lo by a float, corrected once
    const FF<T> an = ff_mul(n, FF<T>{P.alpha[k], P.alpha_lo[k]});
    const T den = eos_denominator(P, k, rho);
    const T r = rcp(den);
    const T q1 = an.hi * r;                                    // within 1.5 ulp
    const FF<T> qd = ff_two_prod(q1, den);
    const T q2 = ((an.hi - qd.hi) - qd.lo + an.lo) * r;       // exact residual / den
    const FF<T> q = ff_two_sum(q1, q2);
    const FF<T> third = {T(1.0 / 3.0), T(1.0 / 3.0 - (double)T(1.0 / 3.0))};
    return ff_mul(ff_add(q, FF<T>{-third.hi, -third.lo}), rho);
}

// psi^k (and the pseudopotential energy U^k = alpha p_EOS - c_s^2 rho) from rho^k.
// Returns true when the square-root argument 2U/g was negative (psi clamped to 0).
// EXACT = false (16-bit population storage, whose rounding is ~2^-11 or coarser)
// evaluates the EOS in plain FP32.
template <bool EXACT = true, typename T>
LBM_HD bool pseudopotential(const Params<T>& P, int k, T rho, T& psi, T& U)
{
    const T g = P.g[k][k];
    if (P.psi_kind[k] == PSI_EOS) {
        if (EXACT && sizeof(T) == 4) {
            const FF<T> u = eos_energy_ff(P, k, rho);
            const FF<T> arg = ff_mul(u, FF<T>{P.two_over_g[k], P.two_over_g_lo[k]});
            U = u.hi + u.lo;
            if (arg.hi <= T(0)) {
                psi = T(0);
                return arg.hi < T(0);
            }
            // sqrt of hi + lo: approximate root from rsqrt, then one Newton step
            // against the exact residual (error ~ the square of the first one's)
            const T ri = rsqrt(arg.hi);
            const T r = arg.hi * ri;
            const FF<T> r2 = ff_two_prod(r, r);
            psi = fma((arg.hi - r2.hi) - r2.lo + arg.lo, T(0.5) * ri, r);
            return false;
        }
        U = P.alpha[k] * eos_pressure(P, k, rho) - rho * T(1.0 / 3.0);
        const T arg = T(2) * U / g;
        psi = sqrt(arg > T(0) ? arg : T(0));
        return arg < T(0);
    }
    psi = P.psi_kind[k] == PSI_RHO ? rho : exp(T(-1) / rho);
    U = T(0.5) * g * psi * psi;
    return false;
}

// ---------------------------------------------------------------------------
// Population storage
// ---------------------------------------------------------------------------
//
// S = T stores the populations themselves. A 16-bit S (FP16 or BF16, FP32
// compute) stores the deviation f_i - w_i rho_ref of component k, rounded to
// nearest; a load adds w_i rho_ref back in FP32.

LBM_HD float pop_to_float(__half v) { return __half2float(v); }
LBM_HD float pop_to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename S>
LBM_HD S pop_from_float(float v);
template <>
LBM_HD __half pop_from_float<__half>(float v) { return __float2half_rn(v); }
template <>
LBM_HD __nv_bfloat16 pop_from_float<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename T, typename S>
constexpr bool pop_shifted = !std::is_same<T, S>::value;

template <class L, typename T, typename S>
LBM_HD T load_pop(const S* __restrict__ p, long long m, int i, T rho_ref)
{
    if constexpr (pop_shifted<T, S>) return pop_to_float(p[m]) + T(L::w(i)) * rho_ref;
    else return p[m];
}

template <class L, typename T, typename S>
LBM_HD void store_pop(S* __restrict__ p, long long m, int i, T v, T rho_ref)
{
    if constexpr (pop_shifted<T, S>) p[m] = pop_from_float<S>(v - T(L::w(i)) * rho_ref);
    else p[m] = v;
}

// The stored value itself: with 16-bit storage the deviation d_i = f_i - w_i rho_ref.
// The density passes need f only through rho = sum_i d_i + rho_ref (the weights sum to
// 1), which saves the shift of every load. The collide pass keeps the shifted loads:
// on the 256^3 PR workload a collide on the deviations measured 3 % slower (0.4366
// against 0.4234 ms per launch), the density pass on them 4.6 % faster (0.1730 against
// 0.1813 ms).
template <typename T, typename S>
LBM_HD T load_raw(const S* __restrict__ p, long long m)
{
    if constexpr (pop_shifted<T, S>) return pop_to_float(p[m]);
    else return p[m];
}

// ---------------------------------------------------------------------------
// Node addressing
// ---------------------------------------------------------------------------

// A node and the slot of its populations: the node index n, or -- on lattices with
// solids, whose populations are stored for fluid nodes only, in fluid-list order --
// its fluid index.
struct Node {
    int x, y, z;
    long long n;
    long long slot = -1;
};

__device__ __forceinline__ bool node_of_thread(int nx, int ny, Node& nd, int z0 = 0)
{
    nd.x = blockIdx.x * blockDim.x + threadIdx.x;
    nd.y = blockIdx.y;
    nd.z = blockIdx.z + z0;
    nd.n = (long long)nd.x + (long long)nx * ((long long)nd.y + (long long)ny * nd.z);
    return nd.x < nx;
}

// Node of this thread in the fluid-node list (lattices with solids): threads map
// to fluid nodes in ascending index order, so solid nodes cost no lanes.
template <typename T>
__device__ __forceinline__ bool node_of_list(const KArgs<T>& a, Node& nd)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_fluid) return false;
    const uint32_t n = (uint32_t)a.fluid[t];
    const uint32_t yz = fast_div(n, a.p.div_nx);
    const uint32_t z = fast_div(yz, a.p.div_ny);
    nd.x = (int)(n - yz * (uint32_t)a.p.nx);
    nd.y = (int)(yz - z * (uint32_t)a.p.ny);
    nd.z = (int)z;
    nd.n = (long long)n;
    nd.slot = t;
    return true;
}

// Node of this thread: from the fluid list when there is one, else from the
// (x, y, z) grid, skipping solid nodes.
template <bool GEOM, typename T>
__device__ __forceinline__ bool fluid_node(const KArgs<T>& a, Node& nd)
{
    if (GEOM && a.fluid) return node_of_list(a, nd);
    if (!node_of_thread(a.p.nx, a.p.ny, nd, a.z0)) return false;
    return !(GEOM && a.solid[nd.n]);
}

// Pull-stream source of direction (ex, ey, ez) at node (x, y, z).
// Returns 0 = regular source *src, 1 = bounce back, 2 = unknown (constant-density face).
template <bool GEOM, typename T>
LBM_HD int pull_source(const Params<T>& P, const uint8_t* __restrict__ solid, int x,
                                           int y, int z, int ex, int ey, int ez, long long& src)
{
    int a = x - ex, b = y - ey, c = z - ez;
    bool wall = false;
    if (a < 0) {
        if (GEOM) {
            if (P.bc[0] == BC_PRESSURE) return 2;
            wall |= P.bc[0] == BC_WALL;
        }
        a += P.nx;
    } else if (a >= P.nx) {
        if (GEOM) {
            if (P.bc[1] == BC_PRESSURE) return 2;
            wall |= P.bc[1] == BC_WALL;
        }
        a -= P.nx;
    }
    if (b < 0) {
        if (GEOM) wall |= P.bc[2] == BC_WALL;
        b += P.ny;
    } else if (b >= P.ny) {
        if (GEOM) wall |= P.bc[3] == BC_WALL;
        b -= P.ny;
    }
    if (c < 0) {
        if (GEOM) wall |= P.bc[4] == BC_WALL;
        c += P.nz;
    } else if (c >= P.nz) {
        if (GEOM) wall |= P.bc[5] == BC_WALL;
        c -= P.nz;
    }
    src = (long long)a + (long long)P.nx * ((long long)b + (long long)P.ny * c);
    if (GEOM && (wall || solid[src])) return 1;
    return 0;
}

// Zou-He / Hecht-Harting closure at a constant-density x face (inward normal
// sign nin): unknown populations have nin * e_x > 0.
//   rho u_n = rho_b - (sum_{e_x = 0} f + 2 sum_{nin e_x < 0} f)
//   f_i = f_opp(i) + 6 w_i rho u_n - (e_iy N_y + e_iz N_z) / 2,  N_t = sum_{e_x = 0} f e_t
// rref != 0: f holds the deviations f_i - w_i rref (16-bit storage); the two face sums
// then take rref times their weight sums, the rest of the closure is unchanged (opposite
// directions share their weight, and the tangential sums of w e vanish)
template <class L, typename T>
LBM_HD void zou_he(T (&f)[L::Q], int nin, T rho_b, T rref = T(0))
{
    T s0 = T(0), sneg = T(0), Ny = T(0), Nz = T(0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int en = L::ex(i) * nin;
        if (en == 0) {
            s0 += f[i];
            if (L::ey(i)) Ny += L::ey(i) > 0 ? f[i] : -f[i];
            if (L::ez(i)) Nz += L::ez(i) > 0 ? f[i] : -f[i];
        } else if (en < 0) {
            sneg += f[i];
        }
    }
    if (rref != T(0)) {
        double w0 = 0.0, wn = 0.0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const int en = L::ex(i) * nin;
            if (en == 0) w0 += L::w(i);
            else if (en < 0) wn += L::w(i);
        }
        s0 = fma(T(w0), rref, s0);
        sneg = fma(T(wn), rref, sneg);
    }
    const T run = rho_b - (s0 + T(2) * sneg);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        if (L::ex(i) * nin > 0) {
            T t = T(0);
            if (L::ey(i)) t += L::ey(i) > 0 ? Ny : -Ny;
            if (L::ez(i)) t += L::ez(i) > 0 ? Nz : -Nz;
            f[i] = f[L::opp(i)] + T(6.0 * L::w(i)) * run - T(0.5) * t;
        }
    }
}

// Periodic lattice without solids: the 3 x 3 x 3 wrapped source offsets of a node
// are formed once, so each of the Q pull sources costs two integer adds (node
// indices fit in 32 bits: the workspace of 2^31 nodes would exceed the HBM).
struct Wrap3 {
    int xo[3], yo[3], zo[3];  // offsets of x - d, d = -1, 0, +1 (index d + 1)
};

template <typename T>
LBM_HD Wrap3 wrap3(const Params<T>& P, int x, int y, int z)
{
    Wrap3 w;
    const int nx = P.nx, ny = P.ny, nz = P.nz, pl = nx * ny;
    w.xo[0] = x == nx - 1 ? 0 : x + 1;       // source x - e with e = -1
    w.xo[1] = x;
    w.xo[2] = x == 0 ? nx - 1 : x - 1;       // e = +1
    w.yo[0] = (y == ny - 1 ? 0 : y + 1) * nx;
    w.yo[1] = y * nx;
    w.yo[2] = (y == 0 ? ny - 1 : y - 1) * nx;
    w.zo[0] = (z == nz - 1 ? 0 : z + 1) * pl;
    w.zo[1] = z * pl;
    w.zo[2] = (z == 0 ? nz - 1 : z - 1) * pl;
    return w;
}

// Per-node neighbour table for every lattice: for each axis the index offsets of the
// coordinates c+1, c, c-1 (index 0, 1, 2, the convention of Wrap3). Periodic axes wrap.
// Across a closed face (wall or constant density) the coordinate is clamped to c, and
// 2 bits of fl record the face kind of that side (1 = wall, 2 = constant density):
// bits [4a, 4a+2) for c+1 leaving through the max face of axis a, [4a+2, 4a+4) for
// c-1 leaving through the min face.
//   pull source of direction e:         offsets [e + 1], face bits of side e + 1
//   force / wetting neighbour x + e:    offsets [1 - e]  (clamped, Section 2.5 stencils)
struct Geo3 {
    int xo[3], yo[3], zo[3];
    unsigned fl;
};

template <bool GEOM, typename T>
LBM_HD Geo3 geo3(const Params<T>& P, int x, int y, int z)
{
    Geo3 g;
    g.fl = 0u;
    if constexpr (!GEOM) {
        const Wrap3 w = wrap3(P, x, y, z);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            g.xo[d] = w.xo[d];
            g.yo[d] = w.yo[d];
            g.zo[d] = w.zo[d];
        }
    } else {
        const int c[3] = {x, y, z}, n[3] = {P.nx, P.ny, P.nz};
        const int stride[3] = {1, P.nx, P.nx * P.ny};
        int* o[3] = {g.xo, g.yo, g.zo};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int bmin = P.bc[2 * a], bmax = P.bc[2 * a + 1];
            o[a][1] = c[a] * stride[a];
            if (c[a] + 1 < n[a]) {
                o[a][0] = (c[a] + 1) * stride[a];
            } else if (bmax == BC_PERIODIC) {
                o[a][0] = 0;
            } else {
                o[a][0] = c[a] * stride[a];
                g.fl |= (bmax == BC_PRESSURE ? 2u : 1u) << (4 * a);
            }
            if (c[a] > 0) {
                o[a][2] = (c[a] - 1) * stride[a];
            } else if (bmin == BC_PERIODIC) {
                o[a][2] = (n[a] - 1) * stride[a];
            } else {
                o[a][2] = c[a] * stride[a];
                g.fl |= (bmin == BC_PRESSURE ? 2u : 1u) << (4 * a + 2);
            }
        }
    }
    return g;
}

// face bits met by the pull source of direction (ex, ey, ez)
LBM_HD unsigned pull_face(const Geo3& g, int ex, int ey, int ez)
{
    unsigned f = 0u;
    if (ex) f |= g.fl >> (ex > 0 ? 2 : 0);
    if (ey) f |= g.fl >> (ey > 0 ? 6 : 4);
    if (ez) f |= g.fl >> (ez > 0 ? 10 : 8);
    return f & 3u;
}

// the direction i with e_i = (ex, ey, ez) (constant-folded for constant arguments)
template <class L>
LBM_HD constexpr int direction_of(int ex, int ey, int ez)
{
    int d = 0;
    for (int i = 0; i < L::Q; ++i)
        if (L::ex(i) == ex && L::ey(i) == ey && L::ez(i) == ez) d = i;
    return d;
}

// index of the force / wetting stencil neighbour x + e
LBM_HD int stencil_index(const Geo3& g, int ex, int ey, int ez)
{
    return g.xo[1 - ex] + g.yo[1 - ey] + g.zo[1 - ez];
}

// Post-stream populations of components k0 .. k0+K-1 at a fluid node (Eq. lbe_steps
// with halfway bounce-back): the pull decision of each direction -- regular source,
// bounce-back at a wall face or solid node, or unknown across a constant-density face
// (completed by Zou-He) -- is taken once and applied to every component.
// With fidx (lattices with solids: fluid-only population storage) a source node m
// holds its populations at slot fidx[m], and fidx[m] < 0 marks a solid.
// DEV (16-bit storage only): f receives the stored deviations (load_raw) instead of the
// populations
template <class L, typename T, typename S, int K, bool GEOM, bool DEV = false>
LBM_HD void gather_all(const void* f_all, const Params<T>& P, const uint8_t* __restrict__ solid,
                       const int* __restrict__ fidx, const Node& nd, const Geo3& g, T (&f)[K][L::Q],
                       int k0 = 0)
{
    constexpr bool RAW = DEV && pop_shifted<T, S>;
    const long long N = P.N;
    const S* fs = static_cast<const S*>(f_all) + (long long)k0 * L::Q * N;
    auto ld = [&](long long m, int i, int k) -> T {
        if constexpr (RAW) return load_raw<T, S>(fs, m);
        else return load_pop<L, T, S>(fs, m, i, P.rho_ref[k0 + k]);
    };
    if constexpr (GEOM && K == 1) {
        if (fidx && g.fl == 0u) {
            // a node on no closed face (almost every node): no pull crosses a face, so a
            // direction is pulled from its source's slot, or bounces back where the slot map
            // marks a solid -- the face logic below reduces to this. One component only: the
            // one-component collide drops its 28 B of spills with it (sphere packs, 17.9 ->
            // 18.5 GLUPS sequential), while the two-component kernels spill more and slow
            // down (porous 400^3: 81.6 -> 71.9 GLUPS)
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const int src = g.xo[L::ex(i) + 1] + g.yo[L::ey(i) + 1] + g.zo[L::ez(i) + 1];
                const int js = i == 0 ? (int)nd.slot : fidx[src];
                const long long m = js < 0 ? (long long)L::opp(i) * N + nd.slot : (long long)i * N + js;
#pragma unroll
                for (int k = 0; k < K; ++k)
                    f[k][i] = ld((long long)k * L::Q * N + m, i, k);
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int src = g.xo[L::ex(i) + 1] + g.yo[L::ey(i) + 1] + g.zo[L::ez(i) + 1];
        if constexpr (!GEOM) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                f[k][i] = ld(((long long)k * L::Q + i) * N + src, i, k);
        } else {
            const unsigned face = i == 0 ? 0u : pull_face(g, L::ex(i), L::ey(i), L::ez(i));
            const bool unknown = (face & 2u) != 0u;   // constant-density x face (precedence)
            long long self, from;
            bool is_solid;
            if (fidx) {
                self = nd.slot;
                const int js = i == 0 ? (int)nd.slot : fidx[src];
                is_solid = js < 0;
                from = js;
            } else {
                self = nd.n;
                is_solid = i != 0 && solid[src];
                from = src;
            }
            const bool bounce = !unknown && (face == 1u || is_solid);
            const long long m = bounce ? (long long)L::opp(i) * N + self : (long long)i * N + from;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const T v = ld((long long)k * L::Q * N + m, i, k);
                f[k][i] = unknown ? T(0) : v;
            }
        }
    }
    if constexpr (GEOM) {
        if (P.bc[0] == BC_PRESSURE && nd.x == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) zou_he<L, T>(f[k], +1, P.bc_rho[0][k0 + k], RAW ? P.rho_ref[k0 + k] : T(0));
        } else if (P.bc[1] == BC_PRESSURE && nd.x == P.nx - 1) {
#pragma unroll
            for (int k = 0; k < K; ++k) zou_he<L, T>(f[k], -1, P.bc_rho[1][k0 + k], RAW ? P.rho_ref[k0 + k] : T(0));
        }
    }
}

template <class L, typename T, typename S, bool GEOM, bool DEV = false>
LBM_HD void gather_k(const void* f_all, const Params<T>& P, const uint8_t* __restrict__ solid, const Node& nd,
                     int k, T (&f)[L::Q], const int* fidx = nullptr)
{
    T fk[1][L::Q];
    gather_all<L, T, S, 1, GEOM, DEV>(f_all, P, solid, fidx, nd, geo3<GEOM>(P, nd.x, nd.y, nd.z), fk, k);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) f[i] = fk[0][i];
}

// rho = sum_i f_i as a balanced tree over opposite-pair sums (rounding error grows
// with the tree depth, log2 Q, instead of with Q for a running sum)
template <class L, typename T>
LBM_HD T density(const T (&f)[L::Q])
{
    constexpr int NP = (L::Q - 1) / 2;
    T s[NP + 1];
    s[0] = f[0];
    static_for<NP>([&](auto pc) {
        constexpr int i = pair_first<L>(decltype(pc)::value);
        constexpr int o = L::opp(i);
        s[decltype(pc)::value + 1] = f[i] + f[o];
    });
#pragma unroll
    for (int w = 1; w < NP + 1; w *= 2)
#pragma unroll
        for (int i = 0; i + w < NP + 1; i += 2 * w) s[i] = s[i] + s[i + w];
    return s[0];
}

template <class L, typename T>
LBM_HD void moments(const T (&f)[L::Q], T& rho, T (&j)[3])
{
    T jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        if (L::opp(i) < i) continue;
        const T d = f[i] - f[L::opp(i)];
        if (L::ex(i)) jx += L::ex(i) > 0 ? d : -d;
        if (L::ey(i)) jy += L::ey(i) > 0 ? d : -d;
        if (L::ez(i)) jz += L::ez(i) > 0 ? d : -d;
    }
    rho = density<L, T>(f);
    j[0] = jx;
    j[1] = jy;
    j[2] = jz;
}

// ---------------------------------------------------------------------------
// Interaction force (Eq. software_ff_force_mcmp), G_i = w_i / c_s^2
// ---------------------------------------------------------------------------

// G_i = w_i / c_s^2 is c_i / 12 with integer c_i (D3Q19: 2 on axis links, 1 on
// edge links; D2Q9: 4 and 1), so the stencil sums integer multiples of neighbour
// differences with compensated summation and scales by 1/12 once. In FP32 this
// keeps the force within about one rounding of its exact value; the force feeds
// the velocity shift F / rho every step, where larger errors grow quickly.
template <class L>
LBM_HD constexpr int g_twelfths(int i)
{
    return (int)(36.0 * L::w(i) + 0.5);  // 12 * 3 w_i
}

// With U^k = g_kk (psi^k)^2 / 2, the pair (i, opp(i)) of Eq. software_ff_force_mcmp
// contributes c_i e_i sum_k' g_kk' dpsi^k' w_kk' with dpsi = psi(x+e_i) - psi(x-e_i),
// w_kk = psi^k(x) + A_k delta^k (delta = mean of the two neighbours minus psi(x)),
// w_kk' = (1 - A_k) psi^k(x) for k' != k. Hence
//   F^k = -(1/12) [ psi^k(x) (g_kk S^k + (1 - A_k) sum_{k'!=k} g_kk' S^k') + A_k g_kk D^k ],
//   S^k = sum_i c_i e_i dpsi^k,
//   D^k = sum_i c_i e_i dpsi^k delta^k (small; accumulated as 2 D^k).
// dpsi is exact whenever the two neighbours lie within a factor of two of each
// other (Sterbenz), which holds across any resolved interface; otherwise its
// rounding is relative to a large difference. The products with psi(x) and g/12
// are formed in double-float: their roundings land on F / rho every step.
// psi_at(k, ex, ey, ez) returns psi^k at x + e (e = 0: at x itself).
// EXACT = false (16-bit population storage) assembles F in plain FP32.
template <class L, typename T, int K, bool EXACT = true, class PsiAt>
LBM_HD void interaction_force_at(const Params<T>& P, const PsiAt& psi_at, const T (&rho)[K], T (&F)[K][3])
{
    T S[K][3], D[K][3], px[K];
    bool mixA[K];   // two components: D^k only enters with A_k != 0 (A_k = 0: Shan-Chen alone)
#pragma unroll
    for (int k = 0; k < K; ++k) {
        px[k] = psi_at(k, 0, 0, 0);
        mixA[k] = K == 1 || P.A[k] != T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) S[k][d] = D[k][d] = T(0);
    }
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        if (L::opp(i) < i) continue;
        const T c = T(g_twelfths<L>(i));
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const T p1 = psi_at(k, L::ex(i), L::ey(i), L::ez(i));
            const T p2 = psi_at(k, -L::ex(i), -L::ey(i), -L::ez(i));
            const T dh = c * (p1 - p2);                            // c <= 4: exact
            if (L::ex(i)) S[k][0] += L::ex(i) > 0 ? dh : -dh;
            if (L::ey(i)) S[k][1] += L::ey(i) > 0 ? dh : -dh;
            if (L::ez(i)) S[k][2] += L::ez(i) > 0 ? dh : -dh;
            if (mixA[k]) {
                const T dd = dh * ((p1 - px[k]) + (p2 - px[k]));   // 2 dpsi delta
                if (L::ex(i)) D[k][0] += L::ex(i) > 0 ? dd : -dd;
                if (L::ey(i)) D[k][1] += L::ey(i) > 0 ? dd : -dd;
                if (L::ez(i)) D[k][2] += L::ez(i) > 0 ? dd : -dd;
            }
        }
    }
    if constexpr (!EXACT) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                T v;
                if (K == 1) {
                    v = P.gm12[k] * fma(px[k], S[k][d], T(0.5) * P.A[k] * D[k][d]);
                } else {
                    T tot = P.g[k][k] * S[k][d];
#pragma unroll
                    for (int kp = 0; kp < K; ++kp)
                        if (kp != k) tot = fma(P.oneA[k] * P.g[k][kp], S[kp][d], tot);
                    v = T(-1.0 / 12.0) * fma(tot, px[k], T(0.5) * P.A[k] * P.g[k][k] * D[k][d]);
                }
                F[k][d] = fma(rho[k], P.accel[k][d], v);
            }
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            FF<T> v;
            if (K == 1) {
                // F = (-g/12) (psi(x) S + A D)
                v = ff_two_prod(px[k], S[k][d]);
                v.lo = fma(T(0.5) * P.A[k], D[k][d], v.lo);
            } else {
                // g_kk S^k + (1 - A_k) sum_{k' != k} g_kk' S^k', times psi^k(x), + A_k g_kk D^k
                FF<T> tot = ff_mul(ff_of(S[k][d]), P.g[k][k]);
#pragma unroll
                for (int kp = 0; kp < K; ++kp) {
                    if (kp == k) continue;
                    tot = ff_add(tot, ff_mul(ff_mul(ff_of(S[kp][d]), P.g[k][kp]), FF<T>{P.oneA[k], P.oneA_lo[k]}));
                }
                v = ff_add(ff_mul(tot, px[k]), ff_of(T(0.5) * P.A[k] * P.g[k][k] * D[k][d]));
            }
            // times -1/12 (K = 1: times -g/12)
            const T ch = K == 1 ? P.gm12[k] : T(-1.0 / 12.0);
            const T cl = K == 1 ? P.gm12_lo[k] : T(-1.0 / 12.0 - (double)T(-1.0 / 12.0));
            const T Fv = fma(v.hi, ch, fma(v.hi, cl, v.lo * ch));
            F[k][d] = fma(rho[k], P.accel[k][d], Fv);
        }
    }
}

// psi read from the global psi array (two-pass step, macroscopic outputs); the
// neighbours come from the node's table g (wrapped, or clamped across closed faces)
template <class L, typename T, int K, bool EXACT = true>
LBM_HD void interaction_force(const KArgs<T>& a, const Node& nd, const Geo3& g, const T (&rho)[K], T (&F)[K][3])
{
    const long long N = a.p.N;
    const T* __restrict__ psi = a.psi;
    auto at = [&](int k, int ex, int ey, int ez) -> T {
        return psi[(long long)k * N + stencil_index(g, ex, ey, ez)];
    };
    interaction_force_at<L, T, K, EXACT>(a.p, at, rho, F);
}

// Moment source C of the surface-tension adjustment (Section 2.3, Eq. mrt_surface and
// Eq. li_surface_adjust) for D2Q9, entries 1, 2, 7, 8 of the moment vector
// (rho, e, eps, jx, qx, jy, qy, pxx, pxy); the rest are zero:
//   C_e = 1.5 s_e (Qxx + Qyy), C_eps = -1.5 s_eps (Qxx + Qyy),
//   C_pxx = -s_nu (Qxx - Qyy), C_pxy = -s_nu Qxy,
//   Q = kappa g_kk/2 [(1 - A) psi(x) sum_i G_i (psi(x+e_i) - psi(x)) e_i e_i
//                     + A/2 sum_i G_i (psi(x+e_i)^2 - psi(x)^2) e_i e_i],
// with the force weights G_i = w_i / c_s^2 and the clamped stencil of the force.
template <class L, typename T, class PsiAt>
LBM_HD void surface_source(const Params<T>& P, const PsiAt& psi_at, int k, T (&C)[L::Q])
{
#pragma unroll
    for (int a = 0; a < L::Q; ++a) C[a] = T(0);
    if (P.kappa_g2[k] == T(0)) return;
    const T px = psi_at(k, 0, 0, 0), A = P.A[k];
    T qxx = T(0), qyy = T(0), qxy = T(0);
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const T pn = psi_at(k, L::ex(i), L::ey(i), L::ez(i));
        const T t = T(3.0 * L::w(i)) * ((T(1) - A) * px * (pn - px) + T(0.5) * A * (pn * pn - px * px));
        if (L::ex(i)) qxx += t;
        if (L::ey(i)) qyy += t;
        if (L::ex(i) && L::ey(i)) qxy += L::ex(i) * L::ey(i) > 0 ? t : -t;
    }
    const T kg = P.kappa_g2[k];
    qxx *= kg;
    qyy *= kg;
    qxy *= kg;
    const T se = P.rates[k][1], seps = P.rates[k][2], snu = P.omega[k];
    C[1] = T(1.5) * se * (qxx + qyy);
    C[2] = T(-1.5) * seps * (qxx + qyy);
    C[7] = -snu * (qxx - qyy);
    C[8] = -snu * qxy;
}

// ---------------------------------------------------------------------------
// Collision (Eq. collision_model) with EDM forcing (Eq. edm)
// ---------------------------------------------------------------------------

// f^eq(rho, u+du) - f^eq(rho, u) for direction i, expanded so that small du
// does not cancel: w rho [3 e.du + 4.5 (e.(2u+du)) (e.du) - 1.5 (2u+du).du]
template <class L, typename T>
LBM_HD T edm_term(int i, T rho, const T (&u)[3], const T (&du)[3])
{
    const T s0 = T(2) * u[0] + du[0], s1 = T(2) * u[1] + du[1], s2 = T(2) * u[2] + du[2];
    T edu = T(0), es = T(0);
    if (L::ex(i)) { edu += L::ex(i) > 0 ? du[0] : -du[0]; es += L::ex(i) > 0 ? s0 : -s0; }
    if (L::ey(i)) { edu += L::ey(i) > 0 ? du[1] : -du[1]; es += L::ey(i) > 0 ? s1 : -s1; }
    if (L::ez(i)) { edu += L::ez(i) > 0 ? du[2] : -du[2]; es += L::ez(i) > 0 ? s2 : -s2; }
    const T sdu = s0 * du[0] + s1 * du[1] + s2 * du[2];
    return T(L::w(i)) * rho * (T(3) * edu + T(4.5) * es * edu - T(1.5) * sdu);
}

template <class L, typename T>
LBM_HD T feq(int i, T rho, const T (&u)[3], T uu)
{
    T eu = T(0);
    if (L::ex(i)) eu += L::ex(i) > 0 ? u[0] : -u[0];
    if (L::ey(i)) eu += L::ey(i) > 0 ? u[1] : -u[1];
    if (L::ez(i)) eu += L::ez(i) > 0 ? u[2] : -u[2];
    return T(L::w(i)) * rho * (T(1) + T(3) * eu + T(4.5) * eu * eu - T(1.5) * uu);
}

// f^eq_i = w_i rho (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u) split as hi + lo, with
// hi the rounded product w_i rho (w_i itself carried as hi + lo). The
// non-equilibrium part f_i - f^eq_i is then formed as (f_i - hi) - lo, where
// f_i - hi is exact for f_i close to w_i rho.
template <class L, typename T>
LBM_HD void feq_split(int i, T rho, const T (&u)[3], T uu, T& hi, T& lo)
{
    T eu = T(0);
    if (L::ex(i)) eu += L::ex(i) > 0 ? u[0] : -u[0];
    if (L::ey(i)) eu += L::ey(i) > 0 ? u[1] : -u[1];
    if (L::ez(i)) eu += L::ez(i) > 0 ? u[2] : -u[2];
    const T poly = fma(eu, fma(T(4.5), eu, T(3)), T(-1.5) * uu);
    const double w = L::w(i);
    const T w_hi = T(w), w_lo = T(w - (double)T(w));
    const FF<T> wr = ff_two_prod(w_hi, rho);
    hi = wr.hi;
    lo = fma(wr.hi, poly, fma(w_lo, rho, wr.lo));
}

// D3Q19 MRT collision with EDM forcing in factored form: the same update as the
// generic moment-space path below (f* = f + M^-1 (Delta m^eq - S m^neq), d'Humieres
// basis), with the transforms written through the sums that several moments share.
//   Forward: even moments are combinations of the rest value n0, the axis-pair sums
//   a_x, a_y, a_z and the edge-pair sums B_xy, B_xz, B_yz (plus xy/yz/xz differences
//   of edge pairs); odd moments of the pair differences.
//   EDM: Delta m^eq needs only rho du and the six rho dq_dd' (dq = u'u' - uu).
//   Backward: the even part of a direction depends only on its class (axis x, y, z or
//   edge plane), the odd part on the pair, so each pair gets ev +- od.
// Non-equilibrium pair sums and differences come straight from f: with
// f^eq_i = W (1 + poly_i) + L (W = w rho rounded, L its rounding error plus w_lo rho),
// poly_{i,opp} = t +- 3 e.u and t = 4.5 (e.u)^2 - 1.5 u.u,
//   neq_i + neq_opp = (f_i - W) + (f_opp - W) - 2 (W t + L)   (f - W exact)
//   neq_i - neq_opp = (f_i - f_opp) - 6 W e.u                (f_i - f_opp exact)
template <typename T>
LBM_HD void collide_mrt_d3q19(const Params<T>& P, int k, T (&f)[19], T rho, const T (&u)[3], const T (&du)[3])
{
    constexpr double w_of[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};  // rest, axis, edge
    const T m15uu = T(-1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    T W[3], Lw[3], W6[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T wh = T(w_of[c]), wl = T(w_of[c] - (double)T(w_of[c]));
        const FF<T> wr = ff_two_prod(wh, rho);
        W[c] = wr.hi;
        Lw[c] = fma(wl, rho, wr.lo);
        W6[c] = T(-6) * wr.hi;
    }
    const T n0 = (f[0] - W[0]) - fma(W[0], m15uu, Lw[0]);
    // pair p = directions (2p+1, 2p+2): +x, +y, +z, +x+y, +x-y, +x+z, +x-z, +y+z, +y-z
    const T eu[9] = {u[0], u[1], u[2], u[0] + u[1], u[0] - u[1], u[0] + u[2], u[0] - u[2], u[1] + u[2], u[1] - u[2]};
    T ps[9], pd[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int c = p < 3 ? 1 : 2;
        const T fi = f[2 * p + 1], fo = f[2 * p + 2];
        const T t = fma(T(4.5) * eu[p], eu[p], m15uu);
        ps[p] = fma(T(-2), fma(W[c], t, Lw[c]), (fi - W[c]) + (fo - W[c]));
        pd[p] = fma(W6[c], eu[p], fi - fo);
    }
    // forward transform (moment rows of the d'Humieres basis, unnormalised)
    const T ayz = ps[1] + ps[2], A = ps[0] + ayz;
    const T Bxy = ps[3] + ps[4], Bxz = ps[5] + ps[6], Byz = ps[7] + ps[8];
    const T Bxyxz = Bxy + Bxz, B = Bxyxz + Byz;
    const T m_e = fma(T(-11), A, fma(T(8), B, T(-30) * n0));       // 19 c^2 - 30
    const T m_eps = fma(T(-4), A, fma(T(12), n0, B));               // (21 c^4 - 53 c^2 + 24) / 2
    const T P9 = fma(T(2), ps[0], -ayz), Q9 = fma(T(-2), Byz, Bxyxz);
    const T m_9 = P9 + Q9, m_10 = fma(T(-2), P9, Q9);                // 3x^2 - c^2, (3c^2 - 5)(...)
    const T R11 = ps[1] - ps[2], S11 = Bxy - Bxz;
    const T m_11 = R11 + S11, m_12 = fma(T(-2), R11, S11);          // y^2 - z^2, (3c^2 - 5)(...)
    const T m_13 = ps[3] - ps[4], m_14 = ps[7] - ps[8], m_15 = ps[5] - ps[6];  // xy, yz, xz
    const T X1 = pd[3] + pd[4], X2 = pd[5] + pd[6];
    const T Y1 = pd[3] - pd[4], Y2 = pd[7] + pd[8];
    const T Z1 = pd[5] - pd[6], Z2 = pd[7] - pd[8];
    const T m_4 = fma(T(-4), pd[0], X1 + X2), m_16 = X1 - X2;       // (5c^2 - 9) x, (y^2 - z^2) x
    const T m_6 = fma(T(-4), pd[1], Y1 + Y2), m_17 = Y2 - Y1;       // (5c^2 - 9) y, (z^2 - x^2) y
    const T m_8 = fma(T(-4), pd[2], Z1 + Z2), m_18 = Z1 - Z2;       // (5c^2 - 9) z, (x^2 - y^2) z
    // Delta m^eq: e 19 rho tr(dq), eps -5.5 rho tr(dq), j rho du, q -2/3 rho du,
    // 3p_xx rho (2 dq_xx - dq_yy - dq_zz) and 3pi_xx -1/2 of it, p_ww rho (dq_yy - dq_zz)
    // and pi_ww -1/2 of it, p_xy, p_yz, p_xz rho dq_xy, rho dq_yz, rho dq_xz
    const T up[3] = {u[0] + du[0], u[1] + du[1], u[2] + du[2]};
    const T dxx = fma(u[0], du[0], du[0] * up[0]), dyy = fma(u[1], du[1], du[1] * up[1]);
    const T dzz = fma(u[2], du[2], du[2] * up[2]), dxy = fma(u[0], du[1], du[0] * up[1]);
    const T dyz = fma(u[1], du[2], du[1] * up[2]), dxz = fma(u[0], du[2], du[0] * up[2]);
    const T dyzs = dyy + dzz;
    const T r_tr = rho * (dxx + dyzs), r_9 = rho * fma(T(2), dxx, -dyzs), r_11 = rho * (dyy - dzz);
    const T* sn = P.rates_n[k];
    // normalised m' = (Delta m^eq - s m^neq) / |M_a|^2
    const T e_ = fma(-sn[1], m_e, T(19.0 / 2394.0) * r_tr);
    const T eps_ = fma(-sn[2], m_eps, T(-5.5 / 252.0) * r_tr);
    const T jx_ = T(0.1) * rho * du[0], jy_ = T(0.1) * rho * du[1], jz_ = T(0.1) * rho * du[2];
    const T qx_ = fma(-sn[4], m_4, T(-1.0 / 60.0) * rho * du[0]);
    const T qy_ = fma(-sn[6], m_6, T(-1.0 / 60.0) * rho * du[1]);
    const T qz_ = fma(-sn[8], m_8, T(-1.0 / 60.0) * rho * du[2]);
    const T p9_ = fma(-sn[9], m_9, T(1.0 / 36.0) * r_9);
    const T p10_ = fma(-sn[10], m_10, T(-1.0 / 144.0) * r_9);
    const T p11_ = fma(-sn[11], m_11, T(1.0 / 12.0) * r_11);
    const T p12_ = fma(-sn[12], m_12, T(-1.0 / 48.0) * r_11);
    const T p13_ = fma(-sn[13], m_13, T(0.25) * (rho * dxy));
    const T p14_ = fma(-sn[14], m_14, T(0.25) * (rho * dyz));
    const T p15_ = fma(-sn[15], m_15, T(0.25) * (rho * dxz));
    const T p16_ = -sn[16] * m_16, p17_ = -sn[17] * m_17, p18_ = -sn[18] * m_18;
    // backward transform M^T m'
    f[0] = f[0] + fma(T(-30), e_, T(12) * eps_);
    {
        const T C = fma(T(-11), e_, T(-4) * eps_);
        const T H = fma(T(-2), p10_, p9_), Wv = fma(T(-2), p12_, p11_);
        const T Tyz = C - H;
        const T ev[3] = {fma(T(2), H, C), Tyz + Wv, Tyz - Wv};
        const T od[3] = {fma(T(-4), qx_, jx_), fma(T(-4), qy_, jy_), fma(T(-4), qz_, jz_)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            f[2 * d + 1] = f[2 * d + 1] + (ev[d] + od[d]);
            f[2 * d + 2] = f[2 * d + 2] + (ev[d] - od[d]);
        }
    }
    {
        const T E0 = fma(T(8), e_, eps_), K9 = p9_ + p10_, K11 = p11_ + p12_;
        const T EK = E0 + K9;
        const T b_xy = EK + K11, b_xz = EK - K11, b_yz = fma(T(-2), K9, E0);
        const T Jx = jx_ + qx_, Jy = jy_ + qy_, Jz = jz_ + qz_;
        const T ev[6] = {b_xy + p13_, b_xy - p13_, b_xz + p15_, b_xz - p15_, b_yz + p14_, b_yz - p14_};
        const T od[6] = {(Jx + Jy) + (p16_ - p17_), (Jx - Jy) + (p16_ + p17_),
                         (Jx + Jz) + (p18_ - p16_), (Jx - Jz) - (p16_ + p18_),
                         (Jy + Jz) + (p17_ - p18_), (Jy - Jz) + (p17_ + p18_)};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            f[2 * q + 7] = f[2 * q + 7] + (ev[q] + od[q]);
            f[2 * q + 8] = f[2 * q + 8] + (ev[q] - od[q]);
        }
    }
}

// BGK collision with EDM forcing over opposite pairs (i, opp(i)). e.u, e.du and
// e.(2u + du) change sign between the two directions of a pair, so the even parts of
// f^eq and of the EDM term are formed once per pair and the odd parts once:
//   f^eq_i = W (1 + P_s + P_a) + L,  P_s = 4.5 (e.u)^2 - 1.5 u.u,  P_a = 3 e.u,
//   edm_i  = W (E_s + E_a),           E_s = 4.5 (e.(2u+du)) (e.du) - 1.5 (2u+du).du,  E_a = 3 e.du,
// with the opposite direction taking -P_a, -E_a. W is w rho rounded and L its rounding
// error plus w_lo rho, so neq = (f - W) - (W poly + L) keeps f - W exact, as in the
// per-direction form, and f* = f + (edm - omega neq) lands one rounding on f.
template <class L, typename T>
LBM_HD void collide_bgk_pairs(const Params<T>& P, int k, T (&f)[L::Q], T rho, const T (&u)[3], const T (&du)[3])
{
    constexpr int NP = (L::Q - 1) / 2;
    const T om = P.omega[k];
    const T m15uu = T(-1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const T s[3] = {fma(T(2), u[0], du[0]), fma(T(2), u[1], du[1]), fma(T(2), u[2], du[2])};
    const T m15sdu = T(-1.5) * (s[0] * du[0] + s[1] * du[1] + s[2] * du[2]);
    auto wsplit = [&](double w, T& W, T& Lw) {
        const T wh = T(w), wl = T(w - (double)T(w));
        const FF<T> wr = ff_two_prod(wh, rho);
        W = wr.hi;
        Lw = fma(wl, rho, wr.lo);
    };
    {
        T W, Lw;
        wsplit(L::w(0), W, Lw);
        const T neq = (f[0] - W) - fma(W, m15uu, Lw);
        f[0] = f[0] + fma(-om, neq, W * m15sdu);
    }
    static_for<NP>([&](auto pc) {
        constexpr int i = pair_first<L>(decltype(pc)::value);
        constexpr int o = L::opp(i);
        T W, Lw;
        wsplit(L::w(i), W, Lw);
        T a = T(0), dl = T(0), sg = T(0);
        if constexpr (L::ex(i) != 0) { a += L::ex(i) > 0 ? u[0] : -u[0]; dl += L::ex(i) > 0 ? du[0] : -du[0]; sg += L::ex(i) > 0 ? s[0] : -s[0]; }
        if constexpr (L::ey(i) != 0) { a += L::ey(i) > 0 ? u[1] : -u[1]; dl += L::ey(i) > 0 ? du[1] : -du[1]; sg += L::ey(i) > 0 ? s[1] : -s[1]; }
        if constexpr (L::ez(i) != 0) { a += L::ez(i) > 0 ? u[2] : -u[2]; dl += L::ez(i) > 0 ? du[2] : -du[2]; sg += L::ez(i) > 0 ? s[2] : -s[2]; }
        const T Ps = fma(T(4.5) * a, a, m15uu), Pa = T(3) * a;
        const T Es = fma(T(4.5) * sg, dl, m15sdu), Ea = T(3) * dl;
        const T neq_i = (f[i] - W) - fma(W, Ps + Pa, Lw);
        const T neq_o = (f[o] - W) - fma(W, Ps - Pa, Lw);
        f[i] = f[i] + fma(-om, neq_i, W * (Es + Ea));
        f[o] = f[o] + fma(-om, neq_o, W * (Es - Ea));
    });
}

// Collision and EDM forcing of one component at one node. The update is formed
// as f_i + (small correction) so that only one rounding lands on f_i. BGK adds
// the EDM shift per direction; MRT adds it in moment space together with the
// relaxation, f* = f + M^-1 (Delta m^eq - S m^neq).
// Cm (may be null): moment source added to the relaxation, f* = f - M^-1 (S m_neq - C)
template <class L, typename T, int COLL>
LBM_HD void collide(const Params<T>& P, int k, T (&f)[L::Q], T rho, const T (&u)[3], const T (&du)[3],
                    const T* Cm = nullptr)
{
    if constexpr (COLL != COLL_BGK && L::Q == 19) {
        collide_mrt_d3q19<T>(P, k, f, rho, u, du);
        return;
    }
    if constexpr (COLL == COLL_BGK) {
        if (!(L::D == 2 && P.forcing_moment)) {
            collide_bgk_pairs<L, T>(P, k, f, rho, u, du);
            return;
        }
    }
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    T neq[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        T hi, lo;
        feq_split<L, T>(i, rho, u, uu, hi, lo);
        neq[i] = (f[i] - hi) - lo;
    }
    if (COLL == COLL_BGK) {
        const T om = P.omega[k];
        if (L::D == 2 && P.forcing_moment) {
            // moment-space forcing: the EDM update minus omega times the quadratic part of
            // f^eq at du / 2, w_i rho (4.5 (e.du / 2)^2 - 1.5 |du / 2|^2)
            const T duu = du[0] * du[0] + du[1] * du[1] + du[2] * du[2];
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                T edu = T(0);
                if (L::ex(i)) edu += L::ex(i) > 0 ? du[0] : -du[0];
                if (L::ey(i)) edu += L::ey(i) > 0 ? du[1] : -du[1];
                if (L::ez(i)) edu += L::ez(i) > 0 ? du[2] : -du[2];
                const T q = T(L::w(i)) * rho * fma(T(1.125) * edu, edu, T(-0.375) * duu);
                f[i] = f[i] + fma(-om, neq[i] + q, edm_term<L, T>(i, rho, u, du));
            }
        } else {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) f[i] = f[i] + fma(-om, neq[i], edm_term<L, T>(i, rho, u, du));
        }
    } else {
        // Moment transforms through opposite pairs (i, opp(i)): moments even under
        // e -> -e see f_0 and the pair sums, odd moments the pair differences, which
        // halves the adds of both transforms. Every coefficient is a compile-time
        // constant of the basis.
        constexpr int NP = (L::Q - 1) / 2;
        T ps[NP], pd[NP];
        static_for<NP>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            constexpr int i = pair_first<L>(p);
            constexpr int o = L::opp(i);
            ps[p] = neq[i] + neq[o];
            pd[p] = neq[i] - neq[o];
        });
        // EDM shift in moment space (velocity products as fused multiply-adds)
        T dq[6], dd[6];
        {
            const T up[3] = {u[0] + du[0], u[1] + du[1], u[2] + du[2]};
            int q = 0;
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int dp = d; dp < 3; ++dp) {
                    dd[q] = T(0.25) * du[d] * du[dp];
                    dq[q++] = fma(u[d], du[dp], du[d] * up[dp]);
                }
        }
        const bool fmom = L::D == 2 && P.forcing_moment;
        T m[L::Q];
        static_for<L::Q>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            // (Delta m^eq_a - s_a m^neq_a) / |row a|^2
            T dm = T(0);
            static_for<3>([&](auto dc) {
                constexpr int d = decltype(dc)::value;
                constexpr double c = d < L::D ? 3.0 * edm_A<L>(a, d) : 0.0;
                if constexpr (c != 0.0) dm = fma(T(c), du[d], dm);
            });
            static_for<6>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                constexpr int d = q < 3 ? 0 : (q < 5 ? 1 : 2);
                constexpr int dp = q < 3 ? q : (q < 5 ? q - 2 : 2);
                constexpr double c = (d < L::D && dp < L::D) ? edm_B<L>(a, d, dp) : 0.0;
                if constexpr (c != 0.0) dm = fma(T(c), dq[q], dm);
            });
            dm = dm * rho;
            constexpr double inv_norm = 1.0 / mrt_norm<L>(a);
            if constexpr (a == 0) {
                m[a] = T(0);  // density: neither relaxed nor shifted (unused below)
            } else if constexpr (L::conserved(a)) {
                m[a] = dm * T(inv_norm);
            } else {
                T acc = T(0);
                if constexpr (mrt_even<L>(a)) {
                    constexpr int c0 = L::M(a, 0);
                    if constexpr (c0 != 0) acc = T(c0) * neq[0];
                    static_for<NP>([&](auto pc) {
                        constexpr int c = L::M(a, pair_first<L>(decltype(pc)::value));
                        if constexpr (c == 1) acc += ps[decltype(pc)::value];
                        else if constexpr (c == -1) acc -= ps[decltype(pc)::value];
                        else if constexpr (c != 0) acc += T(c) * ps[decltype(pc)::value];
                    });
                } else {
                    static_for<NP>([&](auto pc) {
                        constexpr int c = L::M(a, pair_first<L>(decltype(pc)::value));
                        if constexpr (c == 1) acc += pd[decltype(pc)::value];
                        else if constexpr (c == -1) acc -= pd[decltype(pc)::value];
                        else if constexpr (c != 0) acc += T(c) * pd[decltype(pc)::value];
                    });
                }
                const T s = L::stress(a) ? P.omega[k] : P.rates[k][a];
                const T cm = Cm ? Cm[a] : T(0);
                if (fmom) {
                    // moment-space forcing = EDM - S (moments of rho du du / 4): the relaxed
                    // part of the second-order equilibrium shift
                    T dg = T(0);
                    static_for<6>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        constexpr int d = q < 3 ? 0 : (q < 5 ? 1 : 2);
                        constexpr int dp = q < 3 ? q : (q < 5 ? q - 2 : 2);
                        constexpr double c = (d < L::D && dp < L::D) ? edm_B<L>(a, d, dp) : 0.0;
                        if constexpr (c != 0.0) dg = fma(T(c), dd[q], dg);
                    });
                    acc = fma(dg, rho, acc);
                }
                m[a] = (fma(-s, acc, dm) + cm) * T(inv_norm);
            }
        });
        // f* = f + M^-1 (Delta m^eq - S m^neq), M^-1 = M^T diag(1 / row norm)
        T relax[L::Q];
        {
            T acc = T(0);
            static_for<L::Q>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                constexpr int c = (a != 0 && mrt_even<L>(a)) ? L::M(a, 0) : 0;
                if constexpr (c != 0) acc += T(c) * m[a];
            });
            relax[0] = acc;
        }
        static_for<NP>([&](auto pc) {
            constexpr int i = pair_first<L>(decltype(pc)::value);
            T ev = T(0), od = T(0);
            static_for<L::Q>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                constexpr int c = a == 0 ? 0 : L::M(a, i);
                constexpr bool even = mrt_even<L>(a);
                T& t = even ? ev : od;
                if constexpr (c == 1) t += m[a];
                else if constexpr (c == -1) t -= m[a];
                else if constexpr (c != 0) t += T(c) * m[a];
            });
            constexpr int o = L::opp(i);
            relax[i] = ev + od;
            relax[o] = ev - od;
        });
#pragma unroll
        for (int i = 0; i < L::Q; ++i) f[i] = f[i] + relax[i];
    }
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

template <typename T>
LBM_HD bool bad_density(T r)
{
    return !(r > T(0)) || !(r < T(1e30));
}

template <class L, typename T, typename S, int K, bool GEOM>
__device__ __forceinline__ void density_node(const KArgs<T>& a, const Node& nd)
{
    const long long N = a.p.N;
    bool bad = false, clamp = false;
    // 16-bit storage: rho is the sum of the stored deviations plus rho_ref
    constexpr bool DEV = pop_shifted<T, S>;
    T f[K][L::Q];
    gather_all<L, T, S, K, GEOM, DEV>(a.f_src, a.p, a.solid, a.fidx, nd, geo3<GEOM>(a.p, nd.x, nd.y, nd.z), f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const T r = DEV ? density<L, T>(f[k]) + a.p.rho_ref[k] : density<L, T>(f[k]);
        T ps, U;
        clamp |= pseudopotential<!pop_shifted<T, S>>(a.p, k, r, ps, U);
        a.psi[(long long)k * N + nd.n] = ps;
        if (GEOM) a.rho[(long long)k * N + nd.n] = r;
        bad |= bad_density(r);
    }
    if (bad) atomicAdd(a.status + ST_UNSTABLE, 1);
    if (clamp) atomicAdd(a.status + ST_PSI_CLAMP, 1);
}

// two components: at most 64 registers (4 CTAs of 256 per SM); a 48-register cap spilled
// 136 B per thread on lattices with solids and measured 18 % slower
template <class L, typename T, typename S, int K, bool GEOM>
__global__ void __launch_bounds__(256, K == 1 ? 0 : 4) k_density(const KArgs<T> a)
{
    Node nd;
    if (fluid_node<GEOM>(a, nd)) density_node<L, T, S, K, GEOM>(a, nd);
}

// virtual density and psi at boundary solid t (Eq. improved_virtual_density)
template <class L, typename T, int K>
__device__ __forceinline__ void virtual_node(const KArgs<T>& a, int t)
{
    const Params<T>& P = a.p;
    // node indices fit in 32 bits (the workspace of 2^31 nodes would exceed the HBM):
    // the coordinates by the exact multiply-high division of the fluid-list kernels
    const uint32_t s = (uint32_t)a.bsolid[t];
    const uint32_t yz = fast_div(s, P.div_nx);
    const uint32_t zq = fast_div(yz, P.div_ny);
    const int x = (int)(s - yz * (uint32_t)P.nx), y = (int)(yz - zq * (uint32_t)P.ny), z = (int)zq;
    const long long N = P.N;
    // The neighbours come from the per-node offset table of the force stencil (periodic
    // faces wrap, other faces clamp; two adds per neighbour), with their solid flags, once
    // for every component. Each neighbour's density is then loaded whatever its flag (the
    // index is in range) and the flag selects whether the sums take it, so the loads do
    // not wait on the flags. A solid neighbour's value -- which this pass may be writing at
    // the same time, if that solid is a boundary solid too -- is never used. A fluid
    // neighbour is taken as one fused multiply-add, num = fma(w, rho, num).
    const Geo3 g = geo3<true>(P, x, y, z);
    uint32_t m[L::Q];
    uint32_t fl = 0u;   // bit i: neighbour i is fluid
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        m[i] = (uint32_t)stencil_index(g, L::ex(i), L::ey(i), L::ez(i));
        fl |= a.solid[m[i]] ? 0u : (1u << i);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T num = T(0), den = T(0);
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            const T r = a.rho[(long long)k * N + m[i]];
            const bool f = (fl >> i) & 1u;
            num = f ? fma(T(L::w(i)), r, num) : num;
            den = f ? den + T(L::w(i)) : den;
        }
        T r = P.wet_phi[k] * (num / den) - P.wet_drho[k];
        r = r < P.rho_min[k] ? P.rho_min[k] : r;
        r = r > P.rho_max[k] ? P.rho_max[k] : r;
        T ps, U;
        pseudopotential(P, k, r, ps, U);
        a.psi[(long long)k * N + s] = ps;
        a.rho[(long long)k * N + s] = r;
    }
}

// 4 CTAs of 256 per SM (at most 64 registers): the two-component pass at its uncapped 70
// registers (3 CTAs) measured 5 % slower on the porous 400^3 workload (0.163 against 0.155 ms)
template <class L, typename T, int K>
__global__ void __launch_bounds__(256, 4) k_virtual(const KArgs<T> a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.n_bsolid) virtual_node<L, T, K>(a, t);
}

template <class L, typename T, typename S, int K, int COLL, bool GEOM>
__device__ __forceinline__ void collide_node(const KArgs<T>& a, const Node& nd)
{
    const Params<T>& P = a.p;
    const long long N = P.N;
    T f[K][L::Q];
    T rho[K], j[K][3];
    T F[K][3];
    // The force assembly is double-float in FP32 and FP64: at a resting interface the
    // interaction force exceeds a driving body force by orders of magnitude (1e5 in the
    // two-layer channel), and the layer fluxes of that channel after 150 000 steps moved by
    // 1.6e-3 with a plain FP32 assembly (10 % faster on the porous workload, not kept).
    constexpr bool EXF = !pop_shifted<T, S>;
    if constexpr (GEOM && K == 2) {
        // two components with solids: the interaction force first, from psi alone, then the
        // pull; the body force rho a joins once rho is known, as fma(rho, a, F_int) like the
        // path below. Measured 5 % faster than force-after-pull at 400^3 (0.877 against
        // 0.923 ms per launch, general double-float assembly). For one component (sphere
        // packs) the same order measured 2 % slower (64 sphere-pack batch).
        const Geo3 g = geo3<GEOM>(P, nd.x, nd.y, nd.z);
        T Fi[K][3];
        {
            const T zero[K] = {};
            interaction_force<L, T, K, EXF>(a, nd, g, zero, Fi);
        }
        gather_all<L, T, S, K, GEOM>(a.f_src, P, a.solid, a.fidx, nd, g, f);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            moments<L, T>(f[k], rho[k], j[k]);
#pragma unroll
            for (int d = 0; d < 3; ++d) F[k][d] = fma(rho[k], P.accel[k][d], Fi[k][d]);
        }
    } else if constexpr (GEOM) {
        // lattices with solids or closed faces: one table for the pull and the force stencil
        const Geo3 g = geo3<GEOM>(P, nd.x, nd.y, nd.z);
        gather_all<L, T, S, K, GEOM>(a.f_src, P, a.solid, a.fidx, nd, g, f);
#pragma unroll
        for (int k = 0; k < K; ++k) moments<L, T>(f[k], rho[k], j[k]);
        interaction_force<L, T, K, EXF>(a, nd, g, rho, F);
    } else if constexpr (COLL == COLL_BGK) {
        // periodic BGK: psi of the node and of its Q-1 neighbours is loaded before the
        // population gather, so the two sets of loads are in flight together (measured
        // 4 % faster than loading psi after the moments; with the larger MRT collision
        // the extra live registers cost more than that, so MRT keeps the order below)
        const Geo3 g = geo3<GEOM>(P, nd.x, nd.y, nd.z);
        T psiv[K][L::Q];
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int i = 0; i < L::Q; ++i)
                psiv[k][i] = a.psi[(long long)k * N + stencil_index(g, L::ex(i), L::ey(i), L::ez(i))];
        gather_all<L, T, S, K, GEOM>(a.f_src, P, a.solid, a.fidx, nd, g, f);
#pragma unroll
        for (int k = 0; k < K; ++k) moments<L, T>(f[k], rho[k], j[k]);
        auto at = [&](int kk, int ex, int ey, int ez) -> T { return psiv[kk][direction_of<L>(ex, ey, ez)]; };
        interaction_force_at<L, T, K, !pop_shifted<T, S>>(P, at, rho, F);
    } else {
        // periodic: the wrapped offsets are cheap to form again, which keeps them out of
        // the registers live across the moments (64 per thread here)
        gather_all<L, T, S, K, GEOM>(a.f_src, P, a.solid, a.fidx, nd, geo3<GEOM>(P, nd.x, nd.y, nd.z), f);
#pragma unroll
        for (int k = 0; k < K; ++k) moments<L, T>(f[k], rho[k], j[k]);
        interaction_force<L, T, K, !pop_shifted<T, S>>(a, nd, geo3<GEOM>(P, nd.x, nd.y, nd.z), rho, F);
    }
    // surface-tension adjustment (D2Q9 MRT, kappa != 0)
    T Cm[K][L::Q];
    bool use_c = false;
    if constexpr (L::D == 2 && COLL == COLL_MRT) {
        const Geo3 gq = geo3<GEOM>(P, nd.x, nd.y, nd.z);
        auto at = [&](int kk, int ex, int ey, int ez) -> T {
            return a.psi[(long long)kk * N + stencil_index(gq, ex, ey, ez)];
        };
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            surface_source<L, T>(P, at, kk, Cm[kk]);
            use_c |= P.kappa_g2[kk] != T(0);
        }
    }
    T uc[3] = {T(0), T(0), T(0)};
    if (K > 1 && P.common_velocity) {
        T den = T(0);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            den += rho[k] * P.omega[k];
#pragma unroll
            for (int d = 0; d < 3; ++d) uc[d] += j[k][d] * P.omega[k];
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) uc[d] /= den;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T u[3], du[3];
        const T inv = rcp(rho[k]);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            u[d] = (K > 1 && P.common_velocity) ? uc[d] : j[k][d] * inv;
            du[d] = F[k][d] * inv;
        }
        collide<L, T, COLL>(P, k, f[k], rho[k], u, du, use_c ? Cm[k] : nullptr);
        S* dst = static_cast<S*>(a.f_dst) + (long long)k * L::Q * N + (a.fidx ? nd.slot : nd.n);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) store_pop<L, T, S>(dst, (long long)i * N, i, f[k][i], P.rho_ref[k]);
    }
}

// two components: 2 CTAs of 256 per SM (up to 128 registers); a cap of 3 CTAs (80
// registers, 52 B of spills on lattices with solids) measured 7 % slower at 400^3. One
// component: 4 CTAs (64 registers); 3 CTAs on lattices with solids measured 3-10 % slower
// on the 64-sphere-pack batch.
template <class L, typename T, typename S, int K, int COLL, bool GEOM>
__global__ void __launch_bounds__(256, K == 1 ? 4 : 2) k_collide(const KArgs<T> a)
{
    Node nd;
    if (fluid_node<GEOM>(a, nd)) collide_node<L, T, S, K, COLL, GEOM>(a, nd);
}

// Free streaming without collision, forcing or psi: the post-stream populations of
// every fluid node, gathered as the collide pass gathers them, are stored unchanged
// in the destination buffer. Same launch shape and population traffic as the collide
// pass (Q reads and Q writes per component and node) without its arithmetic and its
// psi stencil, so the bandwidth it reaches is the ceiling of that access pattern.
template <class L, typename T, typename S, int K, bool GEOM>
__global__ void __launch_bounds__(256, K == 1 ? 4 : 2) k_stream(const KArgs<T> a)
{
    Node nd;
    if (!fluid_node<GEOM>(a, nd)) return;
    const Params<T>& P = a.p;
    const long long N = P.N;
    T f[K][L::Q];
    gather_all<L, T, S, K, GEOM>(a.f_src, P, a.solid, a.fidx, nd, geo3<GEOM>(P, nd.x, nd.y, nd.z), f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        S* dst = static_cast<S*>(a.f_dst) + (long long)k * L::Q * N + (a.fidx ? nd.slot : nd.n);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) store_pop<L, T, S>(dst, (long long)i * N, i, f[k][i], P.rho_ref[k]);
    }
}

// ---------------------------------------------------------------------------
// Single-pass step for periodic lattices without solids (D3Q19)
// ---------------------------------------------------------------------------
//
// Each CTA owns a TX x TY column tile and marches through a chunk of z planes.
// psi of planes z-1, z, z+1 lives in a three-slot shared-memory ring over the
// tile plus a one-node halo; plane z+1 is recomputed from the pre-stream
// populations (gather -> rho -> EOS) just before plane z is collided, so psi
// never travels through HBM. The collide re-gathers the populations of plane z
// (read from HBM one plane earlier, now L2/L1 resident) and writes the new
// post-collision values. Per lattice update HBM sees one read and one write of
// the Q populations (152 B in FP32) instead of the two-pass 236 B. The
// arithmetic is that of the two-pass kernels, value for value.

template <class L, typename T, typename S, int K>
LBM_HD void psi_of_node(const KArgs<T>& a, int x, int y, int z, T (&out)[K])
{
    Node nd{x, y, z, (long long)x + (long long)a.p.nx * ((long long)y + (long long)a.p.ny * z)};
#pragma unroll
    for (int k = 0; k < K; ++k) {
        // 16-bit storage: rho from the stored deviations, as the density pass forms it
        constexpr bool DEV = pop_shifted<T, S>;
        T f[L::Q];
        gather_k<L, T, S, false, DEV>(a.f_src, a.p, nullptr, nd, k, f);
        T U;
        const T r = DEV ? density<L, T>(f) + a.p.rho_ref[k] : density<L, T>(f);
        pseudopotential<!pop_shifted<T, S>>(a.p, k, r, out[k], U);
    }
}

template <class L, typename T, typename S, int K, int COLL, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) k_fused(const KArgs<T> a, int zchunk)
{
    static_assert(L::D == 3, "the z march needs a 3-D lattice");
    constexpr int HX = TX + 2, HY = TY + 2, PL = HX * HY, NH = 2 * HX + 2 * TY;
    __shared__ T ring[3][K][PL];
    const Params<T>& P = a.p;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, nz);
    const long long N = P.N;

    // psi of one plane over tile + halo into a ring slot (coordinates wrap periodically)
    // coordinates here lie in [-1, 2n): one conditional add or subtract wraps them
    auto wrap = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };
    auto plane = [&](int zp, int slot) {
        const int zw = wrap(zp, nz);
        T v[K];
        psi_of_node<L, T, S, K>(a, wrap(x0 + tx, nx), wrap(y0 + ty, ny), zw, v);
#pragma unroll
        for (int k = 0; k < K; ++k) ring[slot][k][(ty + 1) * HX + tx + 1] = v[k];
        for (int h = tid; h < NH; h += TX * TY) {
            int hx, hy;
            if (h < HX) { hx = h - 1; hy = -1; }
            else if (h < 2 * HX) { hx = h - HX - 1; hy = TY; }
            else if (h < 2 * HX + TY) { hx = -1; hy = h - 2 * HX; }
            else { hx = TX; hy = h - 2 * HX - TY; }
            const int xw = wrap(x0 + hx, nx), yw = wrap(y0 + hy, ny);
            psi_of_node<L, T, S, K>(a, xw, yw, zw, v);
#pragma unroll
            for (int k = 0; k < K; ++k) ring[slot][k][(hy + 1) * HX + hx + 1] = v[k];
        }
    };

    plane(z0 - 1, 0);
    plane(z0, 1);
    for (int z = z0; z < z1; ++z) {
        const int rel = z - z0;
        plane(z + 1, (rel + 2) % 3);
        __syncthreads();
        const int x = x0 + tx, y = y0 + ty;
        if (x < nx && y < ny) {
            Node nd{x, y, z, (long long)x + (long long)nx * ((long long)y + (long long)ny * z)};
            T f[K][L::Q];
            T rho[K], j[K][3];
            bool bad = false;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                gather_k<L, T, S, false>(a.f_src, P, nullptr, nd, k, f[k]);
                moments<L, T>(f[k], rho[k], j[k]);
                bad |= bad_density(rho[k]);
            }
            const int sm = rel % 3, sc = (rel + 1) % 3, sp = (rel + 2) % 3;
            auto at = [&](int k, int ex, int ey, int ez) -> T {
                const int slot = ez < 0 ? sm : (ez > 0 ? sp : sc);
                return ring[slot][k][(ty + 1 + ey) * HX + tx + 1 + ex];
            };
            T F[K][3];
            interaction_force_at<L, T, K, !pop_shifted<T, S>>(P, at, rho, F);
            T uc[3] = {T(0), T(0), T(0)};
            if (K > 1 && P.common_velocity) {
                T den = T(0);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    den += rho[k] * P.omega[k];
#pragma unroll
                    for (int d = 0; d < 3; ++d) uc[d] += j[k][d] * P.omega[k];
                }
#pragma unroll
                for (int d = 0; d < 3; ++d) uc[d] /= den;
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                T u[3], du[3];
                const T inv = rcp(rho[k]);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    u[d] = (K > 1 && P.common_velocity) ? uc[d] : j[k][d] * inv;
                    du[d] = F[k][d] * inv;
                }
                collide<L, T, COLL>(P, k, f[k], rho[k], u, du);
                S* dst = static_cast<S*>(a.f_dst) + (long long)k * L::Q * N + nd.n;
#pragma unroll
                for (int i = 0; i < L::Q; ++i) store_pop<L, T, S>(dst, (long long)i * N, i, f[k][i], P.rho_ref[k]);
            }
            if (bad) atomicAdd(a.status + ST_UNSTABLE, 1);
        }
        __syncthreads();
    }
}

// Post-stream populations F_i(x) (equilibrium of given fields, or given values)
// written into the pre-stream buffer so that the next gather reproduces them:
// f*_i(y) = F_i(y + e_i) for a regular link, F_opp(i)(y) where y + e_i is solid or
// a wall, F_i(y) (unused) across a constant-density face.
template <class L, typename T, typename S, bool GEOM, bool EQ>
__global__ void __launch_bounds__(256) k_unstream(const KArgs<T> a)
{
    Node nd;
    if (!node_of_thread(a.p.nx, a.p.ny, nd)) return;
    const Params<T>& P = a.p;
    const long long N = P.N;
    const T rr = P.rho_ref[a.comp];
    if (a.fidx && a.fidx[nd.n] < 0) return;   // fluid-only storage: solids have no slot
    S* dst = static_cast<S*>(a.f_dst) + (long long)a.comp * L::Q * N + (a.fidx ? a.fidx[nd.n] : nd.n);
    if (GEOM && a.solid[nd.n]) {   // never read; stored as zero deviation
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            store_pop<L, T, S>(dst, (long long)i * N, i, pop_shifted<T, S> ? T(L::w(i)) * rr : T(0), rr);
        return;
    }
    auto value = [&](int i, long long m) -> T {
        if (EQ) {
            const T r = (T)a.in_rho[m];
            T u[3] = {T(0), T(0), T(0)};
            if (a.in_u)
                for (int d = 0; d < L::D; ++d) u[d] = (T)a.in_u[(long long)d * N + m];
            const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            return feq<L, T>(i, r, u, uu);
        }
        return a.in_f[(long long)i * N + m];
    };
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        // the target t = y + e_i pulls direction i from y (pull_source with -e)
        long long t;
        const int kind = pull_source<GEOM>(P, a.solid, nd.x, nd.y, nd.z, -L::ex(i), -L::ey(i), -L::ez(i), t);
        T v;
        if (kind == 0) v = value(i, t);
        else if (kind == 1) v = value(L::opp(i), nd.n);
        else v = value(i, nd.n);
        store_pop<L, T, S>(dst, (long long)i * N, i, v, rr);
    }
}

template <class L, typename T, typename S, bool GEOM>
__global__ void __launch_bounds__(256) k_get_pops(const KArgs<T> a)
{
    Node nd;
    if (!node_of_thread(a.p.nx, a.p.ny, nd)) return;
    const long long N = a.p.N;
    T f[L::Q];
    if (GEOM && a.solid[nd.n]) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) f[i] = T(0);
    } else {
        if (a.fidx) nd.slot = a.fidx[nd.n];
        gather_k<L, T, S, GEOM>(a.f_src, a.p, a.solid, nd, a.comp, f, a.fidx);
    }
#pragma unroll
    for (int i = 0; i < L::Q; ++i) a.out_f[(long long)i * N + nd.n] = f[i];
}

// rho and u = (j + F/2) / rho of one component or of the mixture at one node
template <class L, typename T, typename S, int K, bool GEOM>
LBM_HD void node_macro(const KArgs<T>& a, const Node& nd, int comp, T& r_out,
                                           T (&u_out)[3], T (&rk)[K], T (&mk)[K][3])
{
    const Geo3 g = geo3<GEOM>(a.p, nd.x, nd.y, nd.z);
    T f[K][L::Q];
    T j[K][3];
    gather_all<L, T, S, K, GEOM>(a.f_src, a.p, a.solid, a.fidx, nd, g, f);
#pragma unroll
    for (int k = 0; k < K; ++k) moments<L, T>(f[k], rk[k], j[k]);
    T F[K][3];
    interaction_force<L, T, K, !pop_shifted<T, S>>(a, nd, g, rk, F);
    T r = T(0), m[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int d = 0; d < 3; ++d) mk[k][d] = j[k][d] + T(0.5) * F[k][d];
        if (comp >= 0 && comp != k) continue;
        r += rk[k];
#pragma unroll
        for (int d = 0; d < 3; ++d) m[d] += mk[k][d];
    }
    r_out = r;
#pragma unroll
    for (int d = 0; d < 3; ++d) u_out[d] = m[d] / r;
}

template <class L, typename T, typename S, int K, bool GEOM>
__global__ void __launch_bounds__(256) k_macro(const KArgs<T> a)
{
    Node nd;
    if (!node_of_thread(a.p.nx, a.p.ny, nd)) return;
    const long long N = a.p.N;
    T r = T(0), u[3] = {T(0), T(0), T(0)};
    if (!(GEOM && a.solid[nd.n])) {
        if (a.fidx) nd.slot = a.fidx[nd.n];
        T rk[K], mk[K][3];
        node_macro<L, T, S, K, GEOM>(a, nd, a.comp, r, u, rk, mk);
    }
    if (a.out_rho) a.out_rho[nd.n] = r;
    if (a.out_u)
#pragma unroll
        for (int d = 0; d < L::D; ++d) a.out_u[(long long)d * N + nd.n] = u[d];
}

// Deterministic block reduction of 8 doubles (warp shuffles, then one warp).
__device__ __forceinline__ void block_sum8(double (&v)[8], double* out)
{
    __shared__ double sh[DIAG_THREADS / 32][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 8; ++c) sh[warp][c] = v[c];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            double s = lane < DIAG_THREADS / 32 ? sh[lane][c] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) out[c] = s;
        }
    }
}

// Partial sums per block (fixed grid, grid-stride in node order):
// [0..1] mass per component, [2..7] momentum per component (j + F/2) -- or, in
// residual mode, [0] sum |u - u_prev|^2 and [1] sum |u|^2 of the mixture velocity.
template <class L, typename T, typename S, int K, bool GEOM>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag(const KArgs<T> a)
{
    const Params<T>& P = a.p;
    const long long N = P.N;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long n = (long long)blockIdx.x * DIAG_THREADS + threadIdx.x; n < N;
         n += (long long)DIAG_BLOCKS * DIAG_THREADS) {
        Node nd;
        nd.n = n;
        nd.x = (int)(n % P.nx);
        nd.y = (int)((n / P.nx) % P.ny);
        nd.z = (int)(n / ((long long)P.nx * P.ny));
        if (GEOM && a.solid[n]) continue;
        if (a.fidx) nd.slot = a.fidx[n];
        T r, u[3], rk[K], mk[K][3];
        node_macro<L, T, S, K, GEOM>(a, nd, -1, r, u, rk, mk);
        if (a.want_residual) {
            double du2 = 0.0, uu = 0.0;
#pragma unroll
            for (int d = 0; d < L::D; ++d) {
                const double ud = (double)u[d];
                const double dd = ud - (double)a.u_prev[(long long)d * N + n];
                du2 += dd * dd;
                uu += ud * ud;
                a.u_prev[(long long)d * N + n] = u[d];
            }
            v[0] += du2;
            v[1] += uu;
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                v[k] += (double)rk[k];
#pragma unroll
                for (int d = 0; d < 3; ++d) v[2 + 3 * k + d] += (double)mk[k][d];
            }
        }
    }
    block_sum8(v, a.partials + (long long)blockIdx.x * 8);
}

static __global__ void k_diag_final(const double* __restrict__ partials, double* __restrict__ totals)
{
    // one warp: each lane sums a fixed stride of blocks in order, then a fixed tree
    const int lane = threadIdx.x;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = lane; b < DIAG_BLOCKS; b += 32)
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] += partials[b * 8 + c];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
        if (lane == 0) totals[c] = v[c];
    }
}

// ---------------------------------------------------------------------------
// Batched passes: many lattices in one persistent launch
// ---------------------------------------------------------------------------
//
// The CTAs of every lattice of a batch form one virtual CTA space (each lattice
// needs ceil(units / blockDim) of them: fluid nodes for density / collide,
// boundary solids for the virtual pass). A persistent grid walks that space; a
// CTA finds the lattice of its virtual CTA by binary search over the first
// virtual CTA of each lattice, stages that lattice's kernel arguments in shared
// memory, and runs the same per-node code as the single-lattice kernels.

template <typename T>
__device__ __forceinline__ int batch_item_of(const BatchItem<T>* __restrict__ items, int n, int bop, long long vb)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].vb0[bop] <= vb) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// copy the kernel arguments of one lattice into shared memory (whole CTA)
template <typename T>
__device__ __forceinline__ void stage_args(KArgs<T>& dst, const KArgs<T>& src)
{
    static_assert(sizeof(KArgs<T>) % sizeof(int) == 0, "KArgs is copied in words");
    const int* s = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int w = threadIdx.x; w < (int)(sizeof(KArgs<T>) / sizeof(int)); w += blockDim.x) d[w] = s[w];
}

// node of unit t of a lattice: the t-th fluid node (fluid list) or node t
template <typename T>
__device__ __forceinline__ bool node_of_unit(const KArgs<T>& a, long long t, Node& nd)
{
    uint32_t n;
    if (a.fluid) {
        if (t >= a.n_fluid) return false;
        n = (uint32_t)a.fluid[t];
    } else {
        if (t >= a.p.N) return false;
        n = (uint32_t)t;
    }
    nd.slot = t;
    const uint32_t yz = fast_div(n, a.p.div_nx);
    const uint32_t z = fast_div(yz, a.p.div_ny);
    nd.x = (int)(n - yz * (uint32_t)a.p.nx);
    nd.y = (int)(yz - z * (uint32_t)a.p.ny);
    nd.z = (int)z;
    nd.n = (long long)n;
    return true;
}

template <class L, typename T, typename S, int K, int COLL, bool GEOM, int BOP>
__global__ void __launch_bounds__(256, BOP == BOP_COLLIDE ? (K == 1 ? 4 : 2) : (K == 1 ? 0 : 4))
kb_pass(const BatchItem<T>* __restrict__ items, int n_items, long long nvb, int parity)
{
    __shared__ __align__(16) unsigned char sbuf[sizeof(KArgs<T>)];
    KArgs<T>& sa = *reinterpret_cast<KArgs<T>*>(sbuf);
    int staged = -1;
    for (long long vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        const int s = batch_item_of(items, n_items, BOP, vb);
        if (s != staged) {   // the same for the whole CTA
            __syncthreads();
            stage_args(sa, items[s].a[parity]);
            __syncthreads();
            staged = s;
        }
        const long long t = (vb - items[s].vb0[BOP]) * blockDim.x + threadIdx.x;
        if constexpr (BOP == BOP_VIRTUAL) {
            if (t < sa.n_bsolid) virtual_node<L, T, K>(sa, (int)t);
        } else {
            Node nd;
            if (node_of_unit(sa, t, nd)) {
                if constexpr (BOP == BOP_DENSITY) density_node<L, T, S, K, GEOM>(sa, nd);
                else collide_node<L, T, S, K, COLL, GEOM>(sa, nd);
            }
        }
    }
}

template <class L, typename T, typename S, int K, int COLL, bool GEOM>
cudaError_t run_batch_k(int bop, const BatchItem<T>* items, int n_items, const BatchLaunch& b, int parity,
                        cudaStream_t st)
{
    if (b.nvb <= 0) return cudaSuccess;
    switch (bop) {
    case BOP_DENSITY:
        kb_pass<L, T, S, K, COLL, GEOM, BOP_DENSITY><<<b.grid, b.block, 0, st>>>(items, n_items, b.nvb, parity);
        break;
    case BOP_VIRTUAL:
        kb_pass<L, T, S, K, COLL, GEOM, BOP_VIRTUAL><<<b.grid, b.block, 0, st>>>(items, n_items, b.nvb, parity);
        break;
    case BOP_COLLIDE:
        kb_pass<L, T, S, K, COLL, GEOM, BOP_COLLIDE><<<b.grid, b.block, 0, st>>>(items, n_items, b.nvb, parity);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

inline dim3 node_block(int nx) { return dim3(nx >= 128 ? 128 : ((nx + 31) / 32) * 32, 1, 1); }
inline dim3 node_grid(int nx, int ny, int nz, dim3 b) { return dim3((nx + b.x - 1) / b.x, ny, nz); }

template <class L, typename T, typename S, int K, int COLL, bool GEOM>
cudaError_t run_k(int op, const KArgs<T>& a)
{
    const dim3 b = node_block(a.p.nx), g = node_grid(a.p.nx, a.p.ny, a.p.nz, b);
    // density / collide: one thread per fluid node from the fluid list when there is
    // one, else the (x, y, z) grid (a z range of it for slab schedules)
    const bool list = GEOM && a.fluid;
    const dim3 lb(256, 1, 1), lg((unsigned)((a.n_fluid > 0 ? a.n_fluid : 1) + 255) / 256, 1, 1);
    const dim3 gz = list ? lg : node_grid(a.p.nx, a.p.ny, a.zcount > 0 ? a.zcount : a.p.nz, b);
    const dim3 bz = list ? lb : b;
    switch (op) {
    case OP_DENSITY: k_density<L, T, S, K, GEOM><<<gz, bz, 0, a.stream>>>(a); break;
    case OP_VIRTUAL:
        if (a.n_bsolid > 0) k_virtual<L, T, K><<<(a.n_bsolid + 255) / 256, 256, 0, a.stream>>>(a);
        break;
    case OP_COLLIDE: k_collide<L, T, S, K, COLL, GEOM><<<gz, bz, 0, a.stream>>>(a); break;
    case OP_STREAM: k_stream<L, T, S, K, GEOM><<<gz, bz, 0, a.stream>>>(a); break;
    case OP_FUSED:
        if constexpr (L::D == 3 && !GEOM) {
            constexpr int TX = 32, TY = 8;
            const int zc = a.zchunk > 0 ? a.zchunk : 32;
            const dim3 fb(TX, TY, 1);
            const dim3 fg((a.p.nx + TX - 1) / TX, (a.p.ny + TY - 1) / TY, (a.p.nz + zc - 1) / zc);
            k_fused<L, T, S, K, COLL, TX, TY><<<fg, fb, 0, a.stream>>>(a, zc);
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    case OP_INIT_EQ: k_unstream<L, T, S, GEOM, true><<<g, b, 0, a.stream>>>(a); break;
    case OP_SET_POPS: k_unstream<L, T, S, GEOM, false><<<g, b, 0, a.stream>>>(a); break;
    case OP_GET_POPS: k_get_pops<L, T, S, GEOM><<<g, b, 0, a.stream>>>(a); break;
    case OP_MACRO: k_macro<L, T, S, K, GEOM><<<g, b, 0, a.stream>>>(a); break;
    case OP_DIAG:
        k_diag<L, T, S, K, GEOM><<<DIAG_BLOCKS, DIAG_THREADS, 0, a.stream>>>(a);
        k_diag_final<<<1, 32, 0, a.stream>>>(a.partials, a.totals);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class L, typename T, typename S>
cudaError_t run(int op, const KArgs<T>& a)
{
    const int K = a.p.ncomp;
    const bool mrt = a.p.collision == COLL_MRT;
    if (K == 1) {
        if (mrt)
            return a.geom ? run_k<L, T, S, 1, COLL_MRT, true>(op, a) : run_k<L, T, S, 1, COLL_MRT, false>(op, a);
        return a.geom ? run_k<L, T, S, 1, COLL_BGK, true>(op, a) : run_k<L, T, S, 1, COLL_BGK, false>(op, a);
    }
    if (mrt) return a.geom ? run_k<L, T, S, 2, COLL_MRT, true>(op, a) : run_k<L, T, S, 2, COLL_MRT, false>(op, a);
    return a.geom ? run_k<L, T, S, 2, COLL_BGK, true>(op, a) : run_k<L, T, S, 2, COLL_BGK, false>(op, a);
}

template <class L, typename T, typename S>
cudaError_t run_batch(int bop, const KArgs<T>& shape, const BatchItem<T>* items, int n_items,
                      const BatchLaunch& launch, int parity, cudaStream_t st)
{
    const int K = shape.p.ncomp;
    const bool mrt = shape.p.collision == COLL_MRT, geom = shape.geom != 0;
#define LBM_RB(KK, CC, GG) run_batch_k<L, T, S, KK, CC, GG>(bop, items, n_items, launch, parity, st)
    if (K == 1) {
        if (mrt) return geom ? LBM_RB(1, COLL_MRT, true) : LBM_RB(1, COLL_MRT, false);
        return geom ? LBM_RB(1, COLL_BGK, true) : LBM_RB(1, COLL_BGK, false);
    }
    if (mrt) return geom ? LBM_RB(2, COLL_MRT, true) : LBM_RB(2, COLL_MRT, false);
    return geom ? LBM_RB(2, COLL_BGK, true) : LBM_RB(2, COLL_BGK, false);
#undef LBM_RB
}

}  // namespace lbm
