// C-ABI entry points (include/lbm.h): parameter validation, workspace carving,
// geometry set-up, and the launch sequence of one time step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "args.h"
#include "lattice.cuh"
#include "lbm.h"

using namespace lbm;

struct lbm_ctx {
    lbm_params prm;
    int Q, D;
    long long N;
    size_t elt;             // bytes per compute value (8 for FP64, 4 otherwise)
    int pop_kind;           // population storage: 0 = compute type, 1 = FP16, 2 = BF16 (shifted)
    size_t pop_es;          // bytes per stored population
    void* stage;            // host-transfer staging (16-bit storage), else null: the idle buffer
    char* ws;
    size_t ws_bytes;
    void* fbuf[2];          // population buffers, [K][Q][N]
    int cur;                // buffer holding the pre-stream populations
    void* psi;
    void* rho;
    uint8_t* solid;
    int* bsolid;            // boundary solids, then the fluid node list, in one N-int region
    int n_bsolid;
    int* fluid;
    int n_fluid;
    int* fidx;              // node -> fluid index (-1 at solids); populations of lattices with
                            // solids are stored for fluid nodes only, at that slot
    void* u_prev;
    int* status;
    double* partials;
    double* totals;
    int geom;               // solids present or a non-periodic face
    int any_solid;
    bool faces_open;        // some face is not periodic
    bool init[2];
    bool have_uprev;
    cudaStream_t stream;
    lbm_status sticky;
    long long launches;
    double T[2];
    Params<float> pf;
    Params<double> pd;
    // two-pass overlap: density slabs on sA, collide slabs on sB, forked from and
    // joined back to the caller's stream every step
    int nslab;
    cudaStream_t sA, sB;
    cudaEvent_t ev_fork, ev_join, ev_d[16];
};

// ---------------------------------------------------------------------------
// Critical temperature of an EOS: the isotherm through the critical point has
// dp/drho = d2p/drho2 = 0. Writing p = R T u(rho) - a c(T) s(rho), the two
// conditions give u' s'' - u'' s' = 0 for rho_c and R T_c c(T_c) = a s'/u'. The
// derivatives come from second-order forward-mode (hyper-dual) arithmetic.
// ---------------------------------------------------------------------------

namespace {

struct HD {
    double v, d, dd;  // value, first and second derivative
};
HD operator+(HD a, HD b) { return {a.v + b.v, a.d + b.d, a.dd + b.dd}; }
HD operator-(HD a, HD b) { return {a.v - b.v, a.d - b.d, a.dd - b.dd}; }
HD operator*(HD a, HD b) { return {a.v * b.v, a.d * b.v + a.v * b.d, a.dd * b.v + 2 * a.d * b.d + a.v * b.dd}; }
HD operator/(HD a, HD b)
{
    const double q = a.v / b.v;
    const double qd = (a.d - q * b.d) / b.v;
    const double qdd = (a.dd - 2 * qd * b.d - q * b.dd) / b.v;
    return {q, qd, qdd};
}
HD cst(double c) { return {c, 0, 0}; }

// repulsive part u (p_rep = R T u) and attractive part s (p_att = a c(T) s)
void eos_parts(int eos, double b, double rho, HD& u, HD& s)
{
    const HD r = {rho, 1, 0};
    const HD one = cst(1);
    switch (eos) {
    case EOS_CS: {
        const HD e = cst(b / 4) * r;
        u = r * (one + e + e * e - e * e * e) / ((one - e) * (one - e) * (one - e));
        s = r * r;
        break;
    }
    case EOS_PR:
        u = r / (one - cst(b) * r);
        s = r * r / (one + cst(2 * b) * r - cst(b * b) * r * r);
        break;
    case EOS_VDW:
        u = r / (one - cst(b) * r);
        s = r * r;
        break;
    default:  // RK, RKS
        u = r / (one - cst(b) * r);
        s = r * r / (one + cst(b) * r);
        break;
    }
}

double critical_temperature(int eos, double a, double b, double R)
{
    const double pole = eos == EOS_CS ? 4.0 / b : 1.0 / b;
    auto h = [&](double rho) {
        HD u, s;
        eos_parts(eos, b, rho, u, s);
        return u.d * s.dd - u.dd * s.d;
    };
    // h > 0 at low density, < 0 near the pole: bracket by a scan, then bisect
    double lo = 1e-6 * pole, hi = lo;
    const int n = 4000;
    for (int m = 1; m < n; ++m) {
        const double r = pole * m / n;
        if (h(r) <= 0) { hi = r; break; }
        lo = r;
    }
    if (hi <= lo) return NAN;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (h(mid) > 0) lo = mid; else hi = mid;
    }
    HD u, s;
    eos_parts(eos, b, 0.5 * (lo + hi), u, s);
    const double x = a * s.d / (R * u.d);  // = T_c c(T_c)
    return eos == EOS_RK ? std::pow(x, 2.0 / 3.0) : x;  // RK: c(T) = T^-1/2
}

double eos_alpha(int eos, double omega, double Tr)
{
    if (eos != EOS_PR && eos != EOS_RKS) return 1.0;
    const double m = eos == EOS_PR ? 0.37464 + 1.54226 * omega - 0.26992 * omega * omega
                                   : 0.480 + 1.574 * omega - 0.176 * omega * omega;
    const double s = 1.0 + m * (1.0 - std::sqrt(Tr));
    return s * s;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
    size_t f, psi, rho, solid, bsolid, fidx, uprev, stage, status, partials, totals, total;
};

bool fin(double v) { return std::isfinite(v); }

lbm_status validate(const lbm_params* p)
{
    if (!p) return LBM_ERR_INVALID_ARG;
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) return LBM_ERR_INVALID_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->ny > 65535 || p->nz > 65535) return LBM_ERR_INVALID_ARG;
    if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return LBM_ERR_INVALID_ARG;  // node index in int32
    if (p->lattice == LBM_D2Q9 && p->nz != 1) return LBM_ERR_INVALID_ARG;
    if (p->ncomp != 1 && p->ncomp != 2) return LBM_ERR_INVALID_ARG;
    if (p->real != LBM_FP32 && p->real != LBM_FP64 && p->real != LBM_FP16S && p->real != LBM_BF16S)
        return LBM_ERR_INVALID_ARG;
    if (p->real == LBM_FP16S || p->real == LBM_BF16S)
        for (int k = 0; k < p->ncomp; ++k)
            if (!fin(p->rho_ref[k])) return LBM_ERR_INVALID_ARG;
    if (p->collision != LBM_BGK && p->collision != LBM_MRT) return LBM_ERR_INVALID_ARG;
    if (p->velocity != LBM_UEQ_COMPONENT && p->velocity != LBM_UEQ_COMMON) return LBM_ERR_INVALID_ARG;
    const int nf = p->lattice == LBM_D2Q9 ? 4 : 6;
    for (int f = 0; f < 6; ++f) {
        const int b = p->bc[f];
        if (f >= nf) continue;
        if (b != LBM_BC_PERIODIC && b != LBM_BC_WALL && b != LBM_BC_PRESSURE) return LBM_ERR_INVALID_ARG;
        if (b == LBM_BC_PRESSURE && f >= 2) return LBM_ERR_INVALID_ARG;  // x faces only
    }
    for (int a = 0; a < nf / 2; ++a)  // periodicity is a property of the axis
        if ((p->bc[2 * a] == LBM_BC_PERIODIC) != (p->bc[2 * a + 1] == LBM_BC_PERIODIC)) return LBM_ERR_INVALID_ARG;
    if ((p->bc[0] == LBM_BC_PRESSURE || p->bc[1] == LBM_BC_PRESSURE) && p->nx < 3) return LBM_ERR_INVALID_ARG;
    for (int k = 0; k < p->ncomp; ++k) {
        if (!(p->tau[k] > 0.5) || !fin(p->tau[k])) return LBM_ERR_INVALID_ARG;
        if (p->collision == LBM_MRT)
            for (int m = 0; m < 19; ++m)
                if (!fin(p->mrt_s[k][m]) || p->mrt_s[k][m] < 0 || p->mrt_s[k][m] >= 2) return LBM_ERR_INVALID_ARG;
        const int pk = p->psi_kind[k];
        if (pk != LBM_PSI_EOS && pk != LBM_PSI_RHO && pk != LBM_PSI_EXP) return LBM_ERR_INVALID_ARG;
        if (pk == LBM_PSI_EOS) {
            if (p->eos[k] < LBM_EOS_CS || p->eos[k] > LBM_EOS_RKS) return LBM_ERR_INVALID_ARG;
            if (!(p->eos_a[k] > 0) || !(p->eos_b[k] > 0) || !(p->eos_R[k] > 0) || !(p->T_red[k] > 0))
                return LBM_ERR_INVALID_ARG;
            if (!fin(p->eos_omega[k]) || !fin(p->alpha[k])) return LBM_ERR_INVALID_ARG;
            if (p->g[k][k] == 0.0) return LBM_ERR_INVALID_ARG;
        }
        for (int kp = 0; kp < p->ncomp; ++kp)
            if (!fin(p->g[k][kp])) return LBM_ERR_INVALID_ARG;
        if (!fin(p->A[k]) || !fin(p->wet_phi[k]) || !fin(p->wet_drho[k])) return LBM_ERR_INVALID_ARG;
        if (std::isnan(p->rho_min[k]) || std::isnan(p->rho_max[k]) || p->rho_min[k] > p->rho_max[k])
            return LBM_ERR_INVALID_ARG;
        for (int d = 0; d < 3; ++d)
            if (!fin(p->body_accel[k][d])) return LBM_ERR_INVALID_ARG;
        // a 2-D lattice has no z velocity: a z acceleration would only enter u.u
        if (p->lattice == LBM_D2Q9 && p->body_accel[k][2] != 0.0) return LBM_ERR_INVALID_ARG;
        for (int f = 0; f < 2; ++f)
            if (p->bc[f] == LBM_BC_PRESSURE && !(p->bc_rho[f][k] > 0)) return LBM_ERR_INVALID_ARG;
    }
    if (p->ncomp == 2 && p->g[0][1] != p->g[1][0]) return LBM_ERR_INVALID_ARG;
    for (int k = 0; k < p->ncomp; ++k) {
        if (!fin(p->kappa[k])) return LBM_ERR_INVALID_ARG;
        if (p->kappa[k] != 0.0 && (p->lattice != LBM_D2Q9 || p->collision != LBM_MRT)) return LBM_ERR_INVALID_ARG;
    }
    if (p->forcing != LBM_FORCING_EDM && p->forcing != LBM_FORCING_MOMENT) return LBM_ERR_INVALID_ARG;
    if (p->forcing == LBM_FORCING_MOMENT && p->lattice != LBM_D2Q9) return LBM_ERR_INVALID_ARG;
    if (p->schedule != LBM_SCHEDULE_AUTO && p->schedule != LBM_SCHEDULE_TWO_PASS &&
        p->schedule != LBM_SCHEDULE_SINGLE_PASS && p->schedule != LBM_SCHEDULE_SLAB_OVERLAP)
        return LBM_ERR_INVALID_ARG;
    return LBM_OK;
}

Layout layout_of(const lbm_params* p)
{
    const int Q = p->lattice == LBM_D2Q9 ? 9 : 19;
    const int D = p->lattice == LBM_D2Q9 ? 2 : 3;
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    const size_t e = p->real == LBM_FP64 ? 8 : 4;                       // compute
    const bool half = p->real == LBM_FP16S || p->real == LBM_BF16S;
    const size_t es = half ? 2 : e;                                       // stored population
    const size_t K = (size_t)p->ncomp;
    Layout L;
    size_t off = 0;
    L.f = off;        off += 2 * align256(K * Q * N * es);
    L.psi = off;      off += align256(K * N * e);
    L.rho = off;      off += align256(K * N * e);
    L.solid = off;    off += align256(N);
    L.bsolid = off;   off += align256(N * sizeof(int));
    L.fidx = off;     off += align256(N * sizeof(int));
    L.uprev = off;    off += align256((size_t)D * N * e);
    // host transfers stage in the idle population buffer; 16-bit buffers are too small
    // for (1 + D) N doubles (fields in) or Q N floats (populations in and out)
    L.stage = off;    off += half ? align256(std::max((size_t)(1 + D) * N * 8, (size_t)Q * N * 4)) : 0;
    L.status = off;   off += 256;
    L.partials = off; off += align256(sizeof(double) * 8 * DIAG_BLOCKS);
    L.totals = off;   off += 256;
    L.total = off;
    return L;
}

template <typename T>
void fill_params(const lbm_ctx* c, Params<T>& P)
{
    const lbm_params* p = &c->prm;
    std::memset(&P, 0, sizeof(P));
    P.nx = p->nx; P.ny = p->ny; P.nz = p->nz;
    P.N = c->N;
    P.div_nx = make_fastdiv((uint32_t)p->nx);
    P.div_ny = make_fastdiv((uint32_t)p->ny);
    P.ncomp = p->ncomp;
    P.collision = p->collision == LBM_MRT ? COLL_MRT : COLL_BGK;
    P.common_velocity = p->velocity == LBM_UEQ_COMMON;
    for (int f = 0; f < 6; ++f) P.bc[f] = (c->D == 2 && f >= 4) ? BC_PERIODIC : p->bc[f];
    const bool d2 = p->lattice == LBM_D2Q9;
    for (int k = 0; k < 2; ++k) {
        const int kk = k < p->ncomp ? k : 0;
        P.psi_kind[k] = p->psi_kind[kk];
        P.eos[k] = p->eos[kk];
        P.omega[k] = (T)(1.0 / p->tau[kk]);
        for (int m = 0; m < 19; ++m) {
            const bool cons = d2 ? D2Q9::conserved(m) : D3Q19::conserved(m);
            const bool str = d2 ? D2Q9::stress(m) : D3Q19::stress(m);
            const double s = cons ? 0.0 : (str ? 1.0 / p->tau[kk] : p->mrt_s[kk][m]);
            const int norm = d2 ? (m < 9 ? mrt_norm<D2Q9>(m) : 1) : mrt_norm<D3Q19>(m);
            P.rates[k][m] = (T)s;
            P.rates_n[k][m] = (T)(s / norm);
        }
        P.eos_a[k] = (T)p->eos_a[kk];
        P.eos_b[k] = (T)p->eos_b[kk];
        P.RT[k] = (T)(p->eos_R[kk] * c->T[kk]);
        P.alphaT[k] = (T)eos_alpha(p->eos[kk], p->eos_omega[kk], p->T_red[kk]);
        P.sqrtT[k] = (T)std::sqrt(c->T[kk]);
        P.alpha[k] = (T)p->alpha[kk];
        {
            // p = rho N(rho) / D(rho); coefficients of N in powers of rho
            const double b = p->eos_b[kk], a = p->eos_a[kk], RT = p->eos_R[kk] * c->T[kk];
            const double att = p->eos[kk] == EOS_RK ? a / std::sqrt(c->T[kk])
                                                    : a * eos_alpha(p->eos[kk], p->eos_omega[kk], p->T_red[kk]);
            double cf[5] = {0, 0, 0, 0, 0};
            switch (p->eos[kk]) {
            case EOS_CS: {  // N = RT (1 + e + e^2 - e^3) - a rho (1 - e)^3, e = b rho / 4
                const double B = b / 4.0;
                cf[0] = RT;
                cf[1] = RT * B - a;
                cf[2] = RT * B * B + 3.0 * a * B;
                cf[3] = -RT * B * B * B - 3.0 * a * B * B;
                cf[4] = a * B * B * B;
                break;
            }
            case EOS_PR:  // N = RT (1 + 2 b rho - b^2 rho^2) - att rho (1 - b rho)
                cf[0] = RT; cf[1] = 2.0 * b * RT - att; cf[2] = att * b - RT * b * b;
                break;
            case EOS_VDW:  // N = RT - a rho (1 - b rho)
                cf[0] = RT; cf[1] = -a; cf[2] = a * b;
                break;
            default:  // RK, RKS: N = RT (1 + b rho) - att rho (1 - b rho)
                cf[0] = RT; cf[1] = RT * b - att; cf[2] = att * b;
                break;
            }
            for (int d = 0; d < 5; ++d) {
                P.eos_c[k][d] = (T)cf[d];
                P.eos_c_lo[k][d] = (T)(cf[d] - (double)P.eos_c[k][d]);
            }
            P.alpha_lo[k] = (T)(p->alpha[kk] - (double)P.alpha[k]);
            const double tg = p->g[kk][kk] != 0.0 ? 2.0 / p->g[kk][kk] : 0.0;
            P.two_over_g[k] = (T)tg;
            P.two_over_g_lo[k] = (T)(tg - (double)P.two_over_g[k]);
            const double gm = -p->g[kk][kk] / 12.0;
            P.gm12[k] = (T)gm;
            P.gm12_lo[k] = (T)(gm - (double)P.gm12[k]);
        }
        P.A[k] = (T)p->A[kk];
        P.oneA[k] = (T)(1.0 - p->A[kk]);
        P.oneA_lo[k] = (T)((1.0 - p->A[kk]) - (double)P.oneA[k]);
        for (int kp = 0; kp < 2; ++kp) P.g[k][kp] = (T)p->g[kk][kp < p->ncomp ? kp : 0];
        P.wet_phi[k] = (T)p->wet_phi[kk];
        P.wet_drho[k] = (T)p->wet_drho[kk];
        P.rho_min[k] = (T)p->rho_min[kk];
        P.rho_max[k] = (T)p->rho_max[kk];
        for (int d = 0; d < 3; ++d) P.accel[k][d] = (T)((d2 && d == 2) ? 0.0 : p->body_accel[kk][d]);
        for (int s = 0; s < 2; ++s) P.bc_rho[s][k] = (T)p->bc_rho[s][kk];
        P.rho_ref[k] = (p->real == LBM_FP16S || p->real == LBM_BF16S) ? (T)p->rho_ref[kk] : T(0);
        P.kappa_g2[k] = (T)(p->kappa[kk] * 0.5 * p->g[kk][kk]);
    }
    P.forcing_moment = p->forcing == LBM_FORCING_MOMENT;
}

template <typename T>
KArgs<T> base_args(lbm_ctx* c, const Params<T>& P)
{
    KArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.p = P;
    a.f_src = c->fbuf[c->cur];
    a.f_dst = c->fbuf[c->cur ^ 1];
    a.psi = (T*)c->psi;
    a.rho = (T*)c->rho;
    a.solid = c->solid;
    a.bsolid = c->bsolid;
    a.n_bsolid = c->n_bsolid;
    a.fluid = c->any_solid ? c->fluid : nullptr;
    a.n_fluid = c->any_solid ? c->n_fluid : 0;
    a.fidx = c->any_solid ? c->fidx : nullptr;
    a.geom = c->geom;
    a.status = c->status;
    a.u_prev = (T*)c->u_prev;
    a.partials = c->partials;
    a.totals = c->totals;
    a.stream = c->stream;
    a.comp = 0;
    return a;
}

template <typename T>
cudaError_t dispatch(lbm_ctx* c, int op, const KArgs<T>& a)
{
    cudaError_t e;
    if constexpr (std::is_same<T, float>::value) {
        const bool d2 = c->prm.lattice == LBM_D2Q9;
        if (c->pop_kind == 1) e = d2 ? run<D2Q9, T, __half>(op, a) : run<D3Q19, T, __half>(op, a);
        else if (c->pop_kind == 2) e = d2 ? run<D2Q9, T, __nv_bfloat16>(op, a) : run<D3Q19, T, __nv_bfloat16>(op, a);
        else e = d2 ? run<D2Q9, T, T>(op, a) : run<D3Q19, T, T>(op, a);
    } else {
        e = c->prm.lattice == LBM_D2Q9 ? run<D2Q9, T, T>(op, a) : run<D3Q19, T, T>(op, a);
    }
    if (e == cudaSuccess) {
        if (op == OP_DIAG) c->launches += 2;
        else if (op != OP_VIRTUAL || c->n_bsolid > 0) c->launches += 1;
    }
    return e;
}

lbm_status fail_cuda(lbm_ctx* c, cudaError_t e)
{
    if (e != cudaSuccess) {
        c->sticky = LBM_ERR_CUDA;
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

// rho, psi, U at fluid nodes and boundary solids for the current time level
template <typename T>
cudaError_t fields_pass(lbm_ctx* c, const Params<T>& P)
{
    KArgs<T> a = base_args<T>(c, P);
    cudaError_t e = dispatch<T>(c, OP_DENSITY, a);
    if (e == cudaSuccess && c->n_bsolid > 0) e = dispatch<T>(c, OP_VIRTUAL, a);
    return e;
}

bool use_fused(const lbm_ctx* c)
{
    return c->prm.schedule == LBM_SCHEDULE_SINGLE_PASS && c->D == 3 && !c->geom;
}

// slabs of the overlapped two-pass step (0: run the two passes back to back)
bool use_overlap(const lbm_ctx* c)
{
    return c->prm.schedule == LBM_SCHEDULE_SLAB_OVERLAP && c->nslab >= 2 && !c->any_solid && c->sA && c->sB;
}

template <typename T>
cudaError_t step_overlapped(lbm_ctx* c, const Params<T>& P)
{
    const int S = c->nslab, nz = c->prm.nz;
    cudaError_t e = cudaEventRecord(c->ev_fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->sA, c->ev_fork, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->sB, c->ev_fork, 0);
    KArgs<T> a = base_args<T>(c, P);
    for (int s = 0; s < S && e == cudaSuccess; ++s) {
        a.z0 = (int)((long long)s * nz / S);
        a.zcount = (int)((long long)(s + 1) * nz / S) - a.z0;
        a.stream = c->sA;
        e = dispatch<T>(c, OP_DENSITY, a);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_d[s], c->sA);
    }
    // collide slab s reads psi of slabs s-1, s, s+1 (z wraps): slabs 1 .. S-1 in
    // order, each after density slab min(s+1, S-1); slab 0 (needs slab S-1) last
    for (int j = 0; j < S && e == cudaSuccess; ++j) {
        const int s = j + 1 < S ? j + 1 : 0;
        const int need = (s == 0 || s + 1 >= S) ? S - 1 : s + 1;
        e = cudaStreamWaitEvent(c->sB, c->ev_d[need], 0);
        a.z0 = (int)((long long)s * nz / S);
        a.zcount = (int)((long long)(s + 1) * nz / S) - a.z0;
        a.stream = c->sB;
        if (e == cudaSuccess) e = dispatch<T>(c, OP_COLLIDE, a);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->sB);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    if (e == cudaSuccess) c->cur ^= 1;
    return e;
}

template <typename T>
cudaError_t step_once(lbm_ctx* c, const Params<T>& P)
{
    if (use_overlap(c)) return step_overlapped<T>(c, P);
    if (use_fused(c)) {
        KArgs<T> a = base_args<T>(c, P);
        const cudaError_t e = dispatch<T>(c, OP_FUSED, a);
        if (e == cudaSuccess) c->cur ^= 1;
        return e;
    }
    cudaError_t e = fields_pass<T>(c, P);
    if (e != cudaSuccess) return e;
    KArgs<T> a = base_args<T>(c, P);
    e = dispatch<T>(c, OP_COLLIDE, a);
    if (e == cudaSuccess) c->cur ^= 1;
    return e;
}

lbm_status check_status_word(lbm_ctx* c)
{
    int st[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e);
    if (st[ST_TIMEOUT]) c->sticky = LBM_ERR_TIMEOUT;
    else if (st[ST_UNSTABLE]) c->sticky = LBM_ERR_UNSTABLE;
    return c->sticky;
}

bool ready(const lbm_ctx* c) { return c->init[0] && (c->prm.ncomp < 2 || c->init[1]); }

// host-side neighbour rule of the stencils (periodic wrap, clamp elsewhere)
long long host_nb(const lbm_ctx* c, int x, int y, int z, int ex, int ey, int ez)
{
    const lbm_params* p = &c->prm;
    int v[3] = {x + ex, y + ey, z + ez};
    const int n[3] = {p->nx, p->ny, p->nz};
    for (int a = 0; a < 3; ++a) {
        const bool per = (c->D == 2 && a == 2) || p->bc[2 * a] == LBM_BC_PERIODIC;
        if (v[a] < 0) v[a] = per ? v[a] + n[a] : 0;
        else if (v[a] >= n[a]) v[a] = per ? v[a] - n[a] : n[a] - 1;
    }
    return (long long)v[0] + (long long)p->nx * ((long long)v[1] + (long long)p->ny * v[2]);
}

template <class L>
int build_boundary_list(const lbm_ctx* c, const uint8_t* solid, std::vector<int>& out)
{
    const lbm_params* p = &c->prm;
    out.clear();
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                const long long n = (long long)x + (long long)p->nx * ((long long)y + (long long)p->ny * z);
                if (!solid[n]) continue;
                for (int i = 1; i < L::Q; ++i)
                    if (!solid[host_nb(c, x, y, z, L::ex(i), L::ey(i), L::ez(i))]) {
                        out.push_back((int)n);
                        break;
                    }
            }
    return (int)out.size();
}

// The second population buffer doubles as staging space for host transfers.
void* staging(lbm_ctx* c) { return c->stage ? c->stage : c->fbuf[c->cur ^ 1]; }

}  // namespace

// ---------------------------------------------------------------------------
// Entry points
// ---------------------------------------------------------------------------

extern "C" {

lbm_status lbm_workspace_size(const lbm_params* p, size_t* bytes)
{
    if (!bytes) return LBM_ERR_INVALID_ARG;
    const lbm_status s = validate(p);
    if (s != LBM_OK) return s;
    *bytes = layout_of(p).total;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_params* p, void* d_workspace, size_t bytes, void* stream, lbm_ctx** out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    lbm_status s = validate(p);
    if (s != LBM_OK) return s;
    const Layout L = layout_of(p);
    if (!d_workspace || bytes < L.total || ((uintptr_t)d_workspace & 255)) return LBM_ERR_WORKSPACE;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_INVALID_ARG;
    c->prm = *p;
    c->Q = p->lattice == LBM_D2Q9 ? 9 : 19;
    c->D = p->lattice == LBM_D2Q9 ? 2 : 3;
    c->N = (long long)p->nx * p->ny * p->nz;
    c->elt = p->real == LBM_FP64 ? 8 : 4;
    c->pop_kind = p->real == LBM_FP16S ? 1 : (p->real == LBM_BF16S ? 2 : 0);
    c->pop_es = c->pop_kind ? 2 : c->elt;
    c->ws = (char*)d_workspace;
    c->ws_bytes = bytes;
    const size_t fbytes = align256((size_t)p->ncomp * c->Q * c->N * c->pop_es);
    c->stage = c->pop_kind ? c->ws + L.stage : nullptr;
    c->fbuf[0] = c->ws + L.f;
    c->fbuf[1] = c->ws + L.f + fbytes;
    c->cur = 0;
    c->psi = c->ws + L.psi;
    c->rho = c->ws + L.rho;
    c->solid = (uint8_t*)(c->ws + L.solid);
    c->bsolid = (int*)(c->ws + L.bsolid);
    c->fidx = (int*)(c->ws + L.fidx);
    c->u_prev = c->ws + L.uprev;
    c->status = (int*)(c->ws + L.status);
    c->partials = (double*)(c->ws + L.partials);
    c->totals = (double*)(c->ws + L.totals);
    c->stream = (cudaStream_t)stream;
    c->sticky = LBM_OK;
    c->faces_open = false;
    for (int f = 0; f < (c->D == 2 ? 4 : 6); ++f) c->faces_open |= p->bc[f] != LBM_BC_PERIODIC;
    c->geom = c->faces_open;
    for (int k = 0; k < 2; ++k) {
        c->T[k] = 0.0;
        if (k < p->ncomp && p->psi_kind[k] == LBM_PSI_EOS) {
            const double tc = critical_temperature(p->eos[k], p->eos_a[k], p->eos_b[k], p->eos_R[k]);
            if (!std::isfinite(tc)) { delete c; return LBM_ERR_INVALID_ARG; }
            c->T[k] = p->T_red[k] * tc;
        }
    }
    fill_params<float>(c, c->pf);
    fill_params<double>(c, c->pd);
    cudaError_t e = cudaMemsetAsync(c->solid, 0, (size_t)c->N, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, 256, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { delete c; return LBM_ERR_CUDA; }
    // slab-overlapped two-pass step: about 32 planes per slab, 2 to 16 slabs
    c->nslab = 0;
    if (p->schedule == LBM_SCHEDULE_SLAB_OVERLAP && c->D == 3 && p->nz >= 64) {
        int S = p->nz / 32;
        c->nslab = S < 2 ? 2 : (S > 16 ? 16 : S);
        bool ok = cudaStreamCreateWithFlags(&c->sA, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&c->sB, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
        for (int s = 0; ok && s < c->nslab; ++s)
            ok = cudaEventCreateWithFlags(&c->ev_d[s], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) { lbm_destroy(c); return LBM_ERR_CUDA; }
    }
    *out = c;
    return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx* c, const uint8_t* solid, int where)
{
    if (!c || !solid || (where != LBM_HOST && where != LBM_DEVICE)) return LBM_ERR_INVALID_ARG;
    if (c->sticky != LBM_OK) return c->sticky;
    std::vector<uint8_t> h((size_t)c->N);
    cudaError_t e;
    if (where == LBM_DEVICE) {
        e = cudaMemcpyAsync(h.data(), solid, (size_t)c->N, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return fail_cuda(c, e);
    } else {
        std::memcpy(h.data(), solid, (size_t)c->N);
    }
    c->any_solid = 0;
    for (auto& v : h) {
        v = v ? 1 : 0;
        c->any_solid |= v;
    }
    // boundary solids, then (with solids present) the fluid nodes in ascending order:
    // at most N entries together
    std::vector<int> list;
    c->n_bsolid = c->D == 2 ? build_boundary_list<D2Q9>(c, h.data(), list)
                            : build_boundary_list<D3Q19>(c, h.data(), list);
    c->n_fluid = 0;
    if (c->any_solid)
        for (long long n = 0; n < c->N; ++n)
            if (!h[(size_t)n]) list.push_back((int)n);
    c->n_fluid = (int)list.size() - c->n_bsolid;
    c->fluid = c->bsolid + c->n_bsolid;
    std::vector<int> fidx;
    if (c->any_solid) {
        fidx.assign((size_t)c->N, -1);
        for (int j = 0; j < c->n_fluid; ++j) fidx[(size_t)list[(size_t)(c->n_bsolid + j)]] = j;
    }
    e = cudaMemcpyAsync(c->solid, h.data(), (size_t)c->N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !list.empty())
        e = cudaMemcpyAsync(c->bsolid, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !fidx.empty())
        e = cudaMemcpyAsync(c->fidx, fidx.data(), sizeof(int) * fidx.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e);
    c->geom = c->faces_open || c->any_solid;
    c->init[0] = c->init[1] = false;
    c->have_uprev = false;
    return LBM_OK;
}

}  // extern "C"

namespace {
template <typename T>
lbm_status init_fields_t(lbm_ctx* c, int comp, const double* rho, const double* u, int where, const Params<T>& P)
{
    const double* drho = rho;
    const double* du = u;
    cudaError_t e = cudaSuccess;
    if (where == LBM_HOST) {
        // stage through the idle population buffer (it is at least (1 + D) N doubles)
        double* st = (double*)staging(c);
        e = cudaMemcpyAsync(st, rho, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->stream);
        drho = st;
        if (e == cudaSuccess && u) {
            e = cudaMemcpyAsync(st + c->N, u, sizeof(double) * c->D * c->N, cudaMemcpyHostToDevice, c->stream);
            du = st + c->N;
        }
        if (e != cudaSuccess) return fail_cuda(c, e);
    }
    KArgs<T> a = base_args<T>(c, P);
    a.f_dst = c->fbuf[c->cur];
    a.comp = comp;
    a.in_rho = drho;
    a.in_u = du;
    e = dispatch<T>(c, OP_INIT_EQ, a);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e);
    c->init[comp] = true;
    c->have_uprev = false;
    return LBM_OK;
}
}  // namespace

extern "C" {

lbm_status lbm_init_fields(lbm_ctx* c, int comp, const double* rho, const double* u, int where)
{
    if (!c || !rho || comp < 0 || comp >= c->prm.ncomp || (where != LBM_HOST && where != LBM_DEVICE))
        return LBM_ERR_INVALID_ARG;
    if (c->sticky != LBM_OK) return c->sticky;
    return c->elt == 8 ? init_fields_t<double>(c, comp, rho, u, where, c->pd)
                       : init_fields_t<float>(c, comp, rho, u, where, c->pf);
}

lbm_status lbm_step(lbm_ctx* c, int nsteps)
{
    if (!c || nsteps < 0) return LBM_ERR_INVALID_ARG;
    if (c->sticky != LBM_OK) return c->sticky;
    if (!ready(c)) return LBM_ERR_STATE;
    for (int s = 0; s < nsteps; ++s) {
        const cudaError_t e = c->elt == 8 ? step_once<double>(c, c->pd) : step_once<float>(c, c->pf);
        if (e != cudaSuccess) return fail_cuda(c, e);
    }
    return LBM_OK;
}

}  // extern "C"

namespace {
template <typename T>
lbm_status macro_t(lbm_ctx* c, int comp, void* rho, void* u, int where, const Params<T>& P)
{
    cudaError_t e = fields_pass<T>(c, P);
    if (e != cudaSuccess) return fail_cuda(c, e);
    KArgs<T> a = base_args<T>(c, P);
    a.comp = comp;
    T* st = (T*)staging(c);
    a.out_rho = rho ? (where == LBM_HOST ? st : (T*)rho) : nullptr;
    a.out_u = u ? (where == LBM_HOST ? st + c->N : (T*)u) : nullptr;
    e = dispatch<T>(c, OP_MACRO, a);
    if (e == cudaSuccess && where == LBM_HOST) {
        if (rho) e = cudaMemcpyAsync(rho, st, sizeof(T) * c->N, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && u)
            e = cudaMemcpyAsync(u, st + c->N, sizeof(T) * c->D * c->N, cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e);
    return check_status_word(c);
}
}  // namespace

extern "C" {

lbm_status lbm_macroscopic(lbm_ctx* c, int comp, void* rho, void* u, int where)
{
    if (!c || comp < -1 || comp >= c->prm.ncomp || (where != LBM_HOST && where != LBM_DEVICE))
        return LBM_ERR_INVALID_ARG;
    if (c->sticky != LBM_OK) return c->sticky;
    if (!ready(c)) return LBM_ERR_STATE;
    return c->elt == 8 ? macro_t<double>(c, comp, rho, u, where, c->pd)
                       : macro_t<float>(c, comp, rho, u, where, c->pf);
}

}  // extern "C"

namespace {
template <typename T>
lbm_status diag_t(lbm_ctx* c, double* mass, double* mom, double* residual, const Params<T>& P)
{
    cudaError_t e = fields_pass<T>(c, P);
    if (e != cudaSuccess) return fail_cuda(c, e);
    double tot[8];
    KArgs<T> a = base_args<T>(c, P);
    a.want_residual = 0;
    e = dispatch<T>(c, OP_DIAG, a);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tot, c->totals, sizeof(tot), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e);
    for (int k = 0; k < c->prm.ncomp; ++k) {
        if (mass) mass[k] = tot[k];
        if (mom)
            for (int d = 0; d < 3; ++d) mom[3 * k + d] = tot[2 + 3 * k + d];
    }
    if (residual) {
        a.want_residual = 1;
        e = dispatch<T>(c, OP_DIAG, a);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tot, c->totals, sizeof(tot), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return fail_cuda(c, e);
        *residual = (c->have_uprev && tot[1] > 0) ? std::sqrt(tot[0] / tot[1]) : 1.0;
        c->have_uprev = true;
    }
    return check_status_word(c);
}
}  // namespace

extern "C" {

lbm_status lbm_diagnostics(lbm_ctx* c, double* mass, double* momentum, double* residual)
{
    if (!c) return LBM_ERR_INVALID_ARG;
    if (c->sticky != LBM_OK) return c->sticky;
    if (!ready(c)) return LBM_ERR_STATE;
    return c->elt == 8 ? diag_t<double>(c, mass, momentum, residual, c->pd)
                       : diag_t<float>(c, mass, momentum, residual, c->pf);
}

}  // extern "C"

namespace {
template <typename T>
lbm_status get_pops_t(lbm_ctx* c, int comp, void* f, int where, const Params<T>& P)
{
    KArgs<T> a = base_args<T>(c, P);
    a.comp = comp;
    T* st = (T*)staging(c);
    a.out_f = where == LBM_HOST ? st : (T*)f;
    cudaError_t e = dispatch<T>(c, OP_GET_POPS, a);
    if (e == cudaSuccess && where == LBM_HOST)
        e = cudaMemcpyAsync(f, st, sizeof(T) * c->Q * c->N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return fail_cuda(c, e);
}
template <typename T>
lbm_status set_pops_t(lbm_ctx* c, int comp, const void* f, int where, const Params<T>& P)
{
    KArgs<T> a = base_args<T>(c, P);
    a.comp = comp;
    a.f_dst = c->fbuf[c->cur];
    const T* src = (const T*)f;
    cudaError_t e = cudaSuccess;
    if (where == LBM_HOST) {
        T* st = (T*)staging(c);
        e = cudaMemcpyAsync(st, f, sizeof(T) * c->Q * c->N, cudaMemcpyHostToDevice, c->stream);
        src = st;
    }
    a.in_f = src;
    if (e == cudaSuccess) e = dispatch<T>(c, OP_SET_POPS, a);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e);
    c->init[comp] = true;
    c->have_uprev = false;
    return LBM_OK;
}
}  // namespace

extern "C" {

lbm_status lbm_get_populations(lbm_ctx* c, int comp, void* f, int where)
{
    if (!c || !f || comp < 0 || comp >= c->prm.ncomp || (where != LBM_HOST && where != LBM_DEVICE))
        return LBM_ERR_INVALID_ARG;
    if (c->sticky != LBM_OK) return c->sticky;
    if (!c->init[comp]) return LBM_ERR_STATE;
    return c->elt == 8 ? get_pops_t<double>(c, comp, f, where, c->pd) : get_pops_t<float>(c, comp, f, where, c->pf);
}

lbm_status lbm_set_populations(lbm_ctx* c, int comp, const void* f, int where)
{
    if (!c || !f || comp < 0 || comp >= c->prm.ncomp || (where != LBM_HOST && where != LBM_DEVICE))
        return LBM_ERR_INVALID_ARG;
    if (c->sticky != LBM_OK) return c->sticky;
    return c->elt == 8 ? set_pops_t<double>(c, comp, f, where, c->pd) : set_pops_t<float>(c, comp, f, where, c->pf);
}

lbm_status lbm_velocity_set(const lbm_ctx* c, int* q, int* e, double* w)
{
    if (!c) return LBM_ERR_INVALID_ARG;
    if (q) *q = c->Q;
    for (int i = 0; i < c->Q; ++i) {
        const bool d2 = c->D == 2;
        if (e) {
            e[3 * i + 0] = d2 ? D2Q9::ex(i) : D3Q19::ex(i);
            e[3 * i + 1] = d2 ? D2Q9::ey(i) : D3Q19::ey(i);
            e[3 * i + 2] = d2 ? D2Q9::ez(i) : D3Q19::ez(i);
        }
        if (w) w[i] = d2 ? D2Q9::w(i) : D3Q19::w(i);
    }
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c)
{
    if (!c) return LBM_ERR_INVALID_ARG;
    if (c->sticky != LBM_OK) return c->sticky;
    return check_status_word(c);
}

long long lbm_kernel_launches(const lbm_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"

namespace {
template <typename T>
lbm_status profile_t(lbm_ctx* c, int nsteps, double* ms, long long* nl, const Params<T>& P)
{
    cudaEvent_t ev[4];
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail_cuda(c, cudaErrorUnknown);
    double acc[3] = {0, 0, 0};
    long long cnt[3] = {0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
        KArgs<T> a = base_args<T>(c, P);
        const bool fused = use_fused(c);
        e = cudaEventRecord(ev[0], c->stream);
        if (e == cudaSuccess && !fused) e = dispatch<T>(c, OP_DENSITY, a);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
        if (e == cudaSuccess && !fused && c->n_bsolid > 0) e = dispatch<T>(c, OP_VIRTUAL, a);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], c->stream);
        if (e == cudaSuccess) e = dispatch<T>(c, fused ? OP_FUSED : OP_COLLIDE, a);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3], c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
        if (e != cudaSuccess) break;
        c->cur ^= 1;
        float t;
        for (int k = 0; k < 3; ++k) {
            if ((k == 1 && c->n_bsolid == 0) || (k < 2 && fused)) continue;
            e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            if (e != cudaSuccess) break;
            acc[k] += t;
            cnt[k] += 1;
        }
    }
    for (auto& x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return fail_cuda(c, e);
    for (int k = 0; k < 3; ++k) {
        if (ms) ms[k] = acc[k];
        if (nl) nl[k] = cnt[k];
    }
    return check_status_word(c);
}
template <typename T>
lbm_status stream_probe_t(lbm_ctx* c, int nsteps, double* ms, const Params<T>& P)
{
    cudaEvent_t ev[2];
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail_cuda(c, cudaErrorUnknown);
    double acc = 0.0;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
        KArgs<T> a = base_args<T>(c, P);
        e = cudaEventRecord(ev[0], c->stream);
        if (e == cudaSuccess) e = dispatch<T>(c, OP_STREAM, a);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        if (e != cudaSuccess) break;
        c->cur ^= 1;
        float t = 0.0f;
        e = cudaEventElapsedTime(&t, ev[0], ev[1]);
        acc += t;
    }
    for (auto& x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return fail_cuda(c, e);
    if (ms) *ms = acc;
    return LBM_OK;
}
}  // namespace

extern "C" {

lbm_status lbm_stream_probe(lbm_ctx* c, int nsteps, double* ms)
{
    if (!c || nsteps < 0) return LBM_ERR_INVALID_ARG;
    if (c->sticky != LBM_OK) return c->sticky;
    if (!ready(c)) return LBM_ERR_STATE;
    return c->elt == 8 ? stream_probe_t<double>(c, nsteps, ms, c->pd) : stream_probe_t<float>(c, nsteps, ms, c->pf);
}

lbm_status lbm_profile_step(lbm_ctx* c, int nsteps, double* ms, long long* launches)
{
    if (!c || nsteps < 0) return LBM_ERR_INVALID_ARG;
    if (c->sticky != LBM_OK) return c->sticky;
    if (!ready(c)) return LBM_ERR_STATE;
    return c->elt == 8 ? profile_t<double>(c, nsteps, ms, launches, c->pd)
                       : profile_t<float>(c, nsteps, ms, launches, c->pf);
}

lbm_status lbm_temperature(const lbm_ctx* c, int comp, double* T)
{
    if (!c || !T || comp < 0 || comp >= c->prm.ncomp) return LBM_ERR_INVALID_ARG;
    *T = c->T[comp];
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c)
{
    if (!c) return;
    if (c->sA || c->sB) {
        // outstanding work of the context must finish before its streams go
        if (c->sB) cudaStreamSynchronize(c->sB);
        if (c->sA) cudaStreamSynchronize(c->sA);
    }
    for (int s = 0; s < 16; ++s)
        if (c->ev_d[s]) cudaEventDestroy(c->ev_d[s]);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->sA) cudaStreamDestroy(c->sA);
    if (c->sB) cudaStreamDestroy(c->sB);
    delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many lattices advanced by one persistent launch per pass, two steps
// per CUDA graph replay
// ---------------------------------------------------------------------------

struct lbm_batch {
    std::vector<lbm_ctx*> ctx;
    cudaStream_t stream;      // the caller's stream: uploads, graph replays, direct passes
    cudaStream_t capture;     // private stream the graph is captured on (the legacy default
                              // stream cannot be captured)
    cudaStream_t launch_on;   // where batch_pass enqueues (stream, or capture while capturing)
    char* ws;
    size_t ws_bytes;
    BatchLaunch launch[3];
    std::vector<unsigned char> host;   // item table as last uploaded
    cudaGraphExec_t exec;
    bool graph_ok;
    long long launches;
    int sms;
};

namespace {

size_t batch_item_bytes(const lbm_ctx* c)
{
    return c->elt == 8 ? sizeof(BatchItem<double>) : sizeof(BatchItem<float>);
}

// lattices of one batch share every template parameter of the batched kernels
bool batch_compatible(const lbm_ctx* a, const lbm_ctx* b)
{
    return a->prm.lattice == b->prm.lattice && a->prm.real == b->prm.real && a->prm.ncomp == b->prm.ncomp &&
           a->prm.collision == b->prm.collision && (a->geom != 0) == (b->geom != 0);
}

long long batch_units(const lbm_ctx* c, int bop)
{
    if (bop == BOP_VIRTUAL) return c->n_bsolid;
    return c->any_solid ? c->n_fluid : c->N;
}

template <typename T>
const Params<T>& params_of(const lbm_ctx* c);
template <>
const Params<float>& params_of<float>(const lbm_ctx* c) { return c->pf; }
template <>
const Params<double>& params_of<double>(const lbm_ctx* c) { return c->pd; }

// item table for the current buffers of every lattice and the current CTA sizes
template <typename T>
void batch_table(lbm_batch* b)
{
    const int n = (int)b->ctx.size();
    std::vector<BatchItem<T>> items((size_t)n);
    long long vb[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) {
        lbm_ctx* c = b->ctx[(size_t)i];
        BatchItem<T>& it = items[(size_t)i];
        std::memset(&it, 0, sizeof(it));
        it.a[0] = base_args<T>(c, params_of<T>(c));
        it.a[1] = it.a[0];
        it.a[1].f_src = it.a[0].f_dst;
        it.a[1].f_dst = const_cast<void*>(it.a[0].f_src);
        for (int op = 0; op < 3; ++op) {
            it.vb0[op] = vb[op];
            const long long blk = b->launch[op].block;
            vb[op] += (batch_units(c, op) + blk - 1) / blk;
        }
    }
    for (int op = 0; op < 3; ++op) b->launch[op].nvb = vb[op];
    b->host.assign(reinterpret_cast<unsigned char*>(items.data()),
                   reinterpret_cast<unsigned char*>(items.data()) + sizeof(BatchItem<T>) * (size_t)n);
}

void batch_grid(lbm_batch* b, int op, int ctas_per_sm)
{
    BatchLaunch& l = b->launch[op];
    const long long want = (long long)b->sms * ctas_per_sm;
    l.grid = (int)std::max(1LL, std::min(want, std::max(l.nvb, 1LL)));
}

cudaError_t batch_upload(lbm_batch* b)
{
    return cudaMemcpyAsync(b->ws, b->host.data(), b->host.size(), cudaMemcpyHostToDevice, b->stream);
}

template <typename T>
cudaError_t batch_pass(lbm_batch* b, int op, int parity)
{
    const lbm_ctx* c0 = b->ctx[0];
    const BatchItem<T>* items = reinterpret_cast<const BatchItem<T>*>(b->ws);
    const BatchItem<T>* h = reinterpret_cast<const BatchItem<T>*>(b->host.data());
    const KArgs<T>& shape = h[0].a[0];
    const int n = (int)b->ctx.size();
    const bool d2 = c0->prm.lattice == LBM_D2Q9;
    cudaStream_t st = b->launch_on;
    if constexpr (std::is_same<T, float>::value) {
        if (c0->pop_kind == 1)
            return d2 ? run_batch<D2Q9, T, __half>(op, shape, items, n, b->launch[op], parity, st)
                      : run_batch<D3Q19, T, __half>(op, shape, items, n, b->launch[op], parity, st);
        if (c0->pop_kind == 2)
            return d2 ? run_batch<D2Q9, T, __nv_bfloat16>(op, shape, items, n, b->launch[op], parity, st)
                      : run_batch<D3Q19, T, __nv_bfloat16>(op, shape, items, n, b->launch[op], parity, st);
    }
    return d2 ? run_batch<D2Q9, T, T>(op, shape, items, n, b->launch[op], parity, st)
              : run_batch<D3Q19, T, T>(op, shape, items, n, b->launch[op], parity, st);
}

// one time step of every lattice: density, virtual density at boundary solids, collide
template <typename T>
cudaError_t batch_step(lbm_batch* b, int parity, long long* launches)
{
    cudaError_t e = cudaSuccess;
    for (int op = 0; op < 3 && e == cudaSuccess; ++op) {
        if (b->launch[op].nvb <= 0) continue;
        e = batch_pass<T>(b, op, parity);
        if (e == cudaSuccess && launches) *launches += 1;
    }
    return e;
}

lbm_status batch_fail(lbm_batch* b, cudaError_t e)
{
    for (lbm_ctx* c : b->ctx) c->sticky = LBM_ERR_CUDA;
    (void)e;
    return LBM_ERR_CUDA;
}

template <typename T>
lbm_status batch_step_t(lbm_batch* b, int nsteps)
{
    batch_table<T>(b);
    cudaError_t e = batch_upload(b);
    if (e != cudaSuccess) return batch_fail(b, e);
    long long per_pair = 0;
    for (int op = 0; op < 3; ++op) per_pair += b->launch[op].nvb > 0 ? 2 : 0;
    if (!b->graph_ok && nsteps >= 2) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            b->launch_on = b->capture;
            cudaError_t e1 = batch_step<T>(b, 0, nullptr);
            if (e1 == cudaSuccess) e1 = batch_step<T>(b, 1, nullptr);
            b->launch_on = b->stream;
            e = cudaStreamEndCapture(b->capture, &g);
            if (e == cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return batch_fail(b, e);
        b->graph_ok = true;
    }
    for (int q = 0; q < nsteps / 2 && e == cudaSuccess; ++q) {
        e = cudaGraphLaunch(b->exec, b->stream);
        if (e == cudaSuccess) b->launches += per_pair;
    }
    if (e == cudaSuccess && (nsteps & 1)) {
        e = batch_step<T>(b, 0, &b->launches);
        if (e == cudaSuccess)
            for (lbm_ctx* c : b->ctx) c->cur ^= 1;
    }
    if (e != cudaSuccess) return batch_fail(b, e);
    return LBM_OK;
}

// time `reps` launches of one pass with CUDA events (after one untimed launch)
template <typename T>
float batch_time_pass(lbm_batch* b, int op, int reps, cudaEvent_t e0, cudaEvent_t e1)
{
    batch_table<T>(b);
    if (batch_upload(b) != cudaSuccess) return -1.0f;
    if (batch_pass<T>(b, op, 0) != cudaSuccess) return -1.0f;
    if (cudaEventRecord(e0, b->stream) != cudaSuccess) return -1.0f;
    for (int r = 0; r < reps; ++r)
        if (batch_pass<T>(b, op, 0) != cudaSuccess) return -1.0f;
    if (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0f;
    return ms / reps;
}

template <typename T>
lbm_status batch_autotune_t(lbm_batch* b, int* config)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return batch_fail(b, cudaErrorUnknown);
    }
    static const int blocks[2] = {128, 256};
    static const int per_sm[4] = {2, 4, 8, 16};
    // density first, so that the collide pass is timed on fresh psi
    const int order[3] = {BOP_DENSITY, BOP_VIRTUAL, BOP_COLLIDE};
    lbm_status st = LBM_OK;
    for (int oi = 0; oi < 3 && st == LBM_OK; ++oi) {
        const int op = order[oi];
        float best = -1.0f;
        int bb = b->launch[op].block, bg = 4;
        for (int bi = 0; bi < 2 && st == LBM_OK; ++bi)
            for (int pi = 0; pi < 4; ++pi) {
                b->launch[op].block = blocks[bi];
                batch_table<T>(b);
                if (b->launch[op].nvb <= 0) break;
                batch_grid(b, op, per_sm[pi] * (256 / blocks[bi]));
                const float ms = batch_time_pass<T>(b, op, 3, e0, e1);
                if (ms < 0.0f) { st = batch_fail(b, cudaErrorUnknown); break; }
                if (best < 0.0f || ms < best) { best = ms; bb = blocks[bi]; bg = per_sm[pi] * (256 / blocks[bi]); }
            }
        b->launch[op].block = bb;
        batch_table<T>(b);
        batch_grid(b, op, bg);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBM_OK) return st;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return batch_fail(b, cudaErrorUnknown);
    b->graph_ok = false;   // launch shapes changed: the next step captures again
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (config)
        for (int op = 0; op < 3; ++op) {
            config[2 * op] = b->launch[op].block;
            config[2 * op + 1] = b->launch[op].grid;
        }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_workspace_size(lbm_ctx* const* ctxs, int n, size_t* bytes)
{
    if (!ctxs || n < 1 || !bytes) return LBM_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return LBM_ERR_INVALID_ARG;
        if (!batch_compatible(ctxs[0], ctxs[i])) return LBM_ERR_INVALID_ARG;
    }
    *bytes = align256(batch_item_bytes(ctxs[0]) * (size_t)n);
    return LBM_OK;
}

lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int n, void* d_workspace, size_t bytes, void* stream,
                            lbm_batch** out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    size_t need = 0;
    const lbm_status s = lbm_batch_workspace_size(ctxs, n, &need);
    if (s != LBM_OK) return s;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j)
            if (ctxs[i] == ctxs[j]) return LBM_ERR_INVALID_ARG;   // each lattice once
    if (!d_workspace || bytes < need || ((uintptr_t)d_workspace & 255)) return LBM_ERR_WORKSPACE;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return LBM_ERR_CUDA;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_INVALID_ARG;
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = (cudaStream_t)stream;
    b->launch_on = b->stream;
    if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return LBM_ERR_CUDA;
    }
    b->ws = (char*)d_workspace;
    b->ws_bytes = bytes;
    b->exec = nullptr;
    b->graph_ok = false;
    b->launches = 0;
    b->sms = sms;
    for (int op = 0; op < 3; ++op) b->launch[op].block = 256;
    if (ctxs[0]->elt == 8) batch_table<double>(b);
    else batch_table<float>(b);
    batch_grid(b, BOP_DENSITY, 6);
    batch_grid(b, BOP_VIRTUAL, 6);
    batch_grid(b, BOP_COLLIDE, 4);
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int* config)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    for (lbm_ctx* c : b->ctx) {
        if (c->sticky != LBM_OK) return c->sticky;
        if (!ready(c)) return LBM_ERR_STATE;
    }
    return b->ctx[0]->elt == 8 ? batch_autotune_t<double>(b, config) : batch_autotune_t<float>(b, config);
}

lbm_status lbm_batch_step(lbm_batch* b, int nsteps)
{
    if (!b || nsteps < 0) return LBM_ERR_INVALID_ARG;
    for (lbm_ctx* c : b->ctx) {
        if (c->sticky != LBM_OK) return c->sticky;
        if (!ready(c)) return LBM_ERR_STATE;
    }
    if (nsteps == 0) return LBM_OK;
    return b->ctx[0]->elt == 8 ? batch_step_t<double>(b, nsteps) : batch_step_t<float>(b, nsteps);
}

long long lbm_batch_launches(const lbm_batch* b) { return b ? b->launches : -1; }

void lbm_batch_destroy(lbm_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
}

const char* lbm_status_str(lbm_status s)
{
    switch (s) {
    case LBM_OK: return "LBM_OK";
    case LBM_ERR_INVALID_ARG: return "LBM_ERR_INVALID_ARG";
    case LBM_ERR_WORKSPACE: return "LBM_ERR_WORKSPACE";
    case LBM_ERR_CUDA: return "LBM_ERR_CUDA";
    case LBM_ERR_UNSTABLE: return "LBM_ERR_UNSTABLE";
    case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT";
    case LBM_ERR_STATE: return "LBM_ERR_STATE";
    }
    return "LBM_ERR_UNKNOWN";
}

}  // extern "C"
