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

#include "args.h"
#include "lattice.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Equation of state and pseudopotential (Section 2.2, Eq. eos_potential)
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T eos_pressure(const Params<T>& P, int k, T rho)
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

// psi^k and U^k from rho^k; returns true when the square-root argument was clamped
template <typename T>
__device__ __forceinline__ bool pseudopotential(const Params<T>& P, int k, T rho, T& psi, T& U)
{
    const T g = P.g[k][k];
    if (P.psi_kind[k] == PSI_EOS) {
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
// Node addressing
// ---------------------------------------------------------------------------

struct Node {
    int x, y, z;
    long long n;
};

__device__ __forceinline__ bool node_of_thread(int nx, int ny, Node& nd)
{
    nd.x = blockIdx.x * blockDim.x + threadIdx.x;
    nd.y = blockIdx.y;
    nd.z = blockIdx.z;
    nd.n = (long long)nd.x + (long long)nx * ((long long)nd.y + (long long)ny * nd.z);
    return nd.x < nx;
}

// Stencil neighbour x + e for the force and wetting stencils: periodic faces
// wrap, other faces clamp the coordinate into the domain.
template <bool GEOM, typename T>
__device__ __forceinline__ long long stencil_nb(const Params<T>& P, int x, int y, int z, int ex, int ey,
                                                int ez)
{
    int a = x + ex, b = y + ey, c = z + ez;
    if (a < 0) a = (!GEOM || P.bc[0] == BC_PERIODIC) ? a + P.nx : 0;
    else if (a >= P.nx) a = (!GEOM || P.bc[1] == BC_PERIODIC) ? a - P.nx : P.nx - 1;
    if (b < 0) b = (!GEOM || P.bc[2] == BC_PERIODIC) ? b + P.ny : 0;
    else if (b >= P.ny) b = (!GEOM || P.bc[3] == BC_PERIODIC) ? b - P.ny : P.ny - 1;
    if (c < 0) c = (!GEOM || P.bc[4] == BC_PERIODIC) ? c + P.nz : 0;
    else if (c >= P.nz) c = (!GEOM || P.bc[5] == BC_PERIODIC) ? c - P.nz : P.nz - 1;
    return (long long)a + (long long)P.nx * ((long long)b + (long long)P.ny * c);
}

// Pull-stream source of direction (ex, ey, ez) at node (x, y, z).
// Returns 0 = regular source *src, 1 = bounce back, 2 = unknown (constant-density face).
template <bool GEOM, typename T>
__device__ __forceinline__ int pull_source(const Params<T>& P, const uint8_t* __restrict__ solid, int x,
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
template <class L, typename T>
__device__ __forceinline__ void zou_he(T (&f)[L::Q], int nin, T rho_b)
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

// Post-stream populations of component k at a fluid node (pull + bounce-back +
// constant-density faces).
template <class L, typename T, bool GEOM>
__device__ __forceinline__ void gather_k(const T* __restrict__ f_all, const Params<T>& P,
                                         const uint8_t* __restrict__ solid, const Node& nd, int k,
                                         T (&f)[L::Q])
{
    const T* fk = f_all + (long long)k * L::Q * P.N;
    const long long N = P.N;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        long long src;
        const int kind = pull_source<GEOM>(P, solid, nd.x, nd.y, nd.z, L::ex(i), L::ey(i), L::ez(i), src);
        if (kind == 0) f[i] = fk[(long long)i * N + src];
        else if (kind == 1) f[i] = fk[(long long)L::opp(i) * N + nd.n];
        else f[i] = T(0);
    }
    if (GEOM) {
        if (nd.x == 0 && P.bc[0] == BC_PRESSURE) zou_he<L, T>(f, +1, P.bc_rho[0][k]);
        else if (nd.x == P.nx - 1 && P.bc[1] == BC_PRESSURE) zou_he<L, T>(f, -1, P.bc_rho[1][k]);
    }
}

template <class L, typename T>
__device__ __forceinline__ void moments(const T (&f)[L::Q], T& rho, T (&j)[3])
{
    T r = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        r += f[i];
        if (L::ex(i)) jx += L::ex(i) > 0 ? f[i] : -f[i];
        if (L::ey(i)) jy += L::ey(i) > 0 ? f[i] : -f[i];
        if (L::ez(i)) jz += L::ez(i) > 0 ? f[i] : -f[i];
    }
    rho = r;
    j[0] = jx;
    j[1] = jy;
    j[2] = jz;
}

// ---------------------------------------------------------------------------
// Interaction force (Eq. software_ff_force_mcmp), G_i = w_i / c_s^2
// ---------------------------------------------------------------------------

template <class L, typename T, int K, bool GEOM>
__device__ __forceinline__ void interaction_force(const KArgs<T>& a, const Node& nd, const T (&rho)[K],
                                                  T (&F)[K][3])
{
    const Params<T>& P = a.p;
    const long long N = P.N;
    T sc[K][3], zc[K][3];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int d = 0; d < 3; ++d) sc[k][d] = zc[k][d] = T(0);
    const bool useU = P.needs_U != 0;
    // opposite pairs (i, opp(i)) with i the odd member: accumulate G_i (v_i - v_opp) e_i
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        if (L::opp(i) < i) continue;
        const int o = L::opp(i);
        const long long m1 = stencil_nb<GEOM>(P, nd.x, nd.y, nd.z, L::ex(i), L::ey(i), L::ez(i));
        const long long m2 = stencil_nb<GEOM>(P, nd.x, nd.y, nd.z, L::ex(o), L::ey(o), L::ez(o));
        T ps1[K], ps2[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            ps1[k] = a.psi[(long long)k * N + m1];
            ps2[k] = a.psi[(long long)k * N + m2];
        }
        const T G = T(3.0 * L::w(i));
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T d = T(0);
#pragma unroll
            for (int kp = 0; kp < K; ++kp) d += P.g[k][kp] * (ps1[kp] - ps2[kp]);
            const T gd = G * d;
            if (L::ex(i)) sc[k][0] += L::ex(i) > 0 ? gd : -gd;
            if (L::ey(i)) sc[k][1] += L::ey(i) > 0 ? gd : -gd;
            if (L::ez(i)) sc[k][2] += L::ez(i) > 0 ? gd : -gd;
            if (useU) {
                const T du = G * (a.U[(long long)k * N + m1] - a.U[(long long)k * N + m2]);
                if (L::ex(i)) zc[k][0] += L::ex(i) > 0 ? du : -du;
                if (L::ey(i)) zc[k][1] += L::ey(i) > 0 ? du : -du;
                if (L::ez(i)) zc[k][2] += L::ez(i) > 0 ? du : -du;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const T pk = a.psi[(long long)k * N + nd.n];
        const T Ak = P.A[k];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            T v = (T(1) - Ak) * (-pk * sc[k][d]);
            if (useU) v += Ak * (-zc[k][d]);
            F[k][d] = v + rho[k] * P.accel[k][d];
        }
    }
}

// ---------------------------------------------------------------------------
// Collision (Eq. collision_model) with EDM forcing (Eq. edm)
// ---------------------------------------------------------------------------

// f^eq(rho, u+du) - f^eq(rho, u) for direction i, expanded so that small du
// does not cancel: w rho [3 e.du + 4.5 (e.(2u+du)) (e.du) - 1.5 (2u+du).du]
template <class L, typename T>
__device__ __forceinline__ T edm_term(int i, T rho, const T (&u)[3], const T (&du)[3])
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
__device__ __forceinline__ T feq(int i, T rho, const T (&u)[3], T uu)
{
    T eu = T(0);
    if (L::ex(i)) eu += L::ex(i) > 0 ? u[0] : -u[0];
    if (L::ey(i)) eu += L::ey(i) > 0 ? u[1] : -u[1];
    if (L::ez(i)) eu += L::ez(i) > 0 ? u[2] : -u[2];
    return T(L::w(i)) * rho * (T(1) + T(3) * eu + T(4.5) * eu * eu - T(1.5) * uu);
}

template <class L, typename T, int COLL>
__device__ __forceinline__ void collide(const Params<T>& P, int k, T (&f)[L::Q], T rho, const T (&u)[3],
                                        const T (&du)[3])
{
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (COLL == COLL_BGK) {
        const T om = P.omega[k];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const T fe = feq<L, T>(i, rho, u, uu);
            f[i] = f[i] + om * (fe - f[i]) + edm_term<L, T>(i, rho, u, du);
        }
    } else {
        T neq[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) neq[i] = f[i] - feq<L, T>(i, rho, u, uu);
        T m[L::Q];
#pragma unroll
        for (int a = 0; a < L::Q; ++a) {
            if (L::conserved(a)) { m[a] = T(0); continue; }
            T acc = T(0);
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const int c = L::M(a, i);
                if (c == 1) acc += neq[i];
                else if (c == -1) acc -= neq[i];
                else if (c != 0) acc += T(c) * neq[i];
            }
            const T s = L::stress(a) ? P.omega[k] : P.rates[k][a];
            m[a] = s * acc * T(1.0 / mrt_norm<L>(a));
        }
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            T acc = T(0);
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                if (L::conserved(a)) continue;
                const int c = L::M(a, i);
                if (c == 1) acc += m[a];
                else if (c == -1) acc -= m[a];
                else if (c != 0) acc += T(c) * m[a];
            }
            f[i] = f[i] - acc + edm_term<L, T>(i, rho, u, du);
        }
    }
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ bool bad_density(T r)
{
    return !(r > T(0)) || !(r < T(1e30));
}

template <class L, typename T, int K, bool GEOM>
__global__ void __launch_bounds__(256) k_density(const KArgs<T> a)
{
    Node nd;
    if (!node_of_thread(a.p.nx, a.p.ny, nd)) return;
    if (GEOM && a.solid[nd.n]) return;
    const long long N = a.p.N;
    bool bad = false, clamp = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T f[L::Q];
        gather_k<L, T, GEOM>(a.f_src, a.p, a.solid, nd, k, f);
        T r = T(0);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) r += f[i];
        T ps, U;
        clamp |= pseudopotential(a.p, k, r, ps, U);
        a.psi[(long long)k * N + nd.n] = ps;
        if (a.p.needs_U) a.U[(long long)k * N + nd.n] = U;
        if (GEOM) a.rho[(long long)k * N + nd.n] = r;
        bad |= bad_density(r);
    }
    if (bad) atomicAdd(a.status + ST_UNSTABLE, 1);
    if (clamp) atomicAdd(a.status + ST_PSI_CLAMP, 1);
}

template <class L, typename T, int K>
__global__ void __launch_bounds__(256) k_virtual(const KArgs<T> a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_bsolid) return;
    const Params<T>& P = a.p;
    const long long s = a.bsolid[t];
    const int x = (int)(s % P.nx), y = (int)((s / P.nx) % P.ny), z = (int)(s / ((long long)P.nx * P.ny));
    const long long N = P.N;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T num = T(0), den = T(0);
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            const long long m = stencil_nb<true>(P, x, y, z, L::ex(i), L::ey(i), L::ez(i));
            if (a.solid[m]) continue;
            num += T(L::w(i)) * a.rho[(long long)k * N + m];
            den += T(L::w(i));
        }
        T r = P.wet_phi[k] * (num / den) - P.wet_drho[k];
        r = r < P.rho_min[k] ? P.rho_min[k] : r;
        r = r > P.rho_max[k] ? P.rho_max[k] : r;
        T ps, U;
        pseudopotential(P, k, r, ps, U);
        a.psi[(long long)k * N + s] = ps;
        if (P.needs_U) a.U[(long long)k * N + s] = U;
        a.rho[(long long)k * N + s] = r;
    }
}

template <class L, typename T, int K, int COLL, bool GEOM>
__global__ void __launch_bounds__(256) k_collide(const KArgs<T> a)
{
    Node nd;
    if (!node_of_thread(a.p.nx, a.p.ny, nd)) return;
    if (GEOM && a.solid[nd.n]) return;
    const Params<T>& P = a.p;
    const long long N = P.N;
    T f[K][L::Q];
    T rho[K], j[K][3];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        gather_k<L, T, GEOM>(a.f_src, P, a.solid, nd, k, f[k]);
        moments<L, T>(f[k], rho[k], j[k]);
    }
    T F[K][3];
    interaction_force<L, T, K, GEOM>(a, nd, rho, F);
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
        const T inv = T(1) / rho[k];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            u[d] = (K > 1 && P.common_velocity) ? uc[d] : j[k][d] * inv;
            du[d] = F[k][d] * inv;
        }
        collide<L, T, COLL>(P, k, f[k], rho[k], u, du);
        T* dst = a.f_dst + (long long)k * L::Q * N + nd.n;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) dst[(long long)i * N] = f[k][i];
    }
}

// Post-stream populations F_i(x) (equilibrium of given fields, or given values)
// written into the pre-stream buffer so that the next gather reproduces them:
// f*_i(y) = F_i(y + e_i) for a regular link, F_opp(i)(y) where y + e_i is solid or
// a wall, F_i(y) (unused) across a constant-density face.
template <class L, typename T, bool GEOM, bool EQ>
__global__ void __launch_bounds__(256) k_unstream(const KArgs<T> a)
{
    Node nd;
    if (!node_of_thread(a.p.nx, a.p.ny, nd)) return;
    const Params<T>& P = a.p;
    const long long N = P.N;
    T* dst = a.f_dst + (long long)a.comp * L::Q * N + nd.n;
    if (GEOM && a.solid[nd.n]) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) dst[(long long)i * N] = T(0);
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
        dst[(long long)i * N] = v;
    }
}

template <class L, typename T, bool GEOM>
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
        gather_k<L, T, GEOM>(a.f_src, a.p, a.solid, nd, a.comp, f);
    }
#pragma unroll
    for (int i = 0; i < L::Q; ++i) a.out_f[(long long)i * N + nd.n] = f[i];
}

// rho and u = (j + F/2) / rho of one component or of the mixture at one node
template <class L, typename T, int K, bool GEOM>
__device__ __forceinline__ void node_macro(const KArgs<T>& a, const Node& nd, int comp, T& r_out,
                                           T (&u_out)[3], T (&rk)[K], T (&mk)[K][3])
{
    T f[L::Q];
    T j[K][3];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        gather_k<L, T, GEOM>(a.f_src, a.p, a.solid, nd, k, f);
        moments<L, T>(f, rk[k], j[k]);
    }
    T F[K][3];
    interaction_force<L, T, K, GEOM>(a, nd, rk, F);
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

template <class L, typename T, int K, bool GEOM>
__global__ void __launch_bounds__(256) k_macro(const KArgs<T> a)
{
    Node nd;
    if (!node_of_thread(a.p.nx, a.p.ny, nd)) return;
    const long long N = a.p.N;
    T r = T(0), u[3] = {T(0), T(0), T(0)};
    if (!(GEOM && a.solid[nd.n])) {
        T rk[K], mk[K][3];
        node_macro<L, T, K, GEOM>(a, nd, a.comp, r, u, rk, mk);
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
template <class L, typename T, int K, bool GEOM>
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
        T r, u[3], rk[K], mk[K][3];
        node_macro<L, T, K, GEOM>(a, nd, -1, r, u, rk, mk);
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
// Launchers
// ---------------------------------------------------------------------------

inline dim3 node_block(int nx) { return dim3(nx >= 256 ? 256 : ((nx + 31) / 32) * 32, 1, 1); }
inline dim3 node_grid(int nx, int ny, int nz, dim3 b) { return dim3((nx + b.x - 1) / b.x, ny, nz); }

template <class L, typename T, int K, int COLL, bool GEOM>
cudaError_t run_k(int op, const KArgs<T>& a)
{
    const dim3 b = node_block(a.p.nx), g = node_grid(a.p.nx, a.p.ny, a.p.nz, b);
    switch (op) {
    case OP_DENSITY: k_density<L, T, K, GEOM><<<g, b, 0, a.stream>>>(a); break;
    case OP_VIRTUAL:
        if (a.n_bsolid > 0) k_virtual<L, T, K><<<(a.n_bsolid + 255) / 256, 256, 0, a.stream>>>(a);
        break;
    case OP_COLLIDE: k_collide<L, T, K, COLL, GEOM><<<g, b, 0, a.stream>>>(a); break;
    case OP_INIT_EQ: k_unstream<L, T, GEOM, true><<<g, b, 0, a.stream>>>(a); break;
    case OP_SET_POPS: k_unstream<L, T, GEOM, false><<<g, b, 0, a.stream>>>(a); break;
    case OP_GET_POPS: k_get_pops<L, T, GEOM><<<g, b, 0, a.stream>>>(a); break;
    case OP_MACRO: k_macro<L, T, K, GEOM><<<g, b, 0, a.stream>>>(a); break;
    case OP_DIAG:
        k_diag<L, T, K, GEOM><<<DIAG_BLOCKS, DIAG_THREADS, 0, a.stream>>>(a);
        k_diag_final<<<1, 32, 0, a.stream>>>(a.partials, a.totals);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class L, typename T>
cudaError_t run(int op, const KArgs<T>& a)
{
    const int K = a.p.ncomp;
    const bool mrt = a.p.collision == COLL_MRT;
    if (K == 1) {
        if (mrt) return a.geom ? run_k<L, T, 1, COLL_MRT, true>(op, a) : run_k<L, T, 1, COLL_MRT, false>(op, a);
        return a.geom ? run_k<L, T, 1, COLL_BGK, true>(op, a) : run_k<L, T, 1, COLL_BGK, false>(op, a);
    }
    if (mrt) return a.geom ? run_k<L, T, 2, COLL_MRT, true>(op, a) : run_k<L, T, 2, COLL_MRT, false>(op, a);
    return a.geom ? run_k<L, T, 2, COLL_BGK, true>(op, a) : run_k<L, T, 2, COLL_BGK, false>(op, a);
}

}  // namespace lbm
