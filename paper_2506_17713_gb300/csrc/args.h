// Kernel argument block shared by the C-ABI layer and the kernel translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm {

enum : int { PSI_EOS = 0, PSI_RHO = 1, PSI_EXP = 2 };
enum : int { EOS_CS = 0, EOS_PR = 1, EOS_VDW = 2, EOS_RK = 3, EOS_RKS = 4 };
enum : int { BC_PERIODIC = 0, BC_WALL = 1, BC_PRESSURE = 2 };
enum : int { COLL_BGK = 0, COLL_MRT = 1 };

// status word slots (device int[8])
enum : int { ST_UNSTABLE = 0, ST_PSI_CLAMP = 1, ST_TIMEOUT = 2 };

// Exact unsigned 32-bit division by an invariant divisor d (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Fig. 4.1):
// with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
//   n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0),  t = mulhi(m, n).
struct FastDiv {
    uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    FastDiv f;
    f.d = d;
    f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

__host__ __device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv& f)
{
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(f.m, n);
#else
    const uint32_t t = (uint32_t)(((uint64_t)f.m * n) >> 32);
#endif
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Physical parameters in the compute type T, resolved on the host.
template <typename T>
struct Params {
    int nx, ny, nz;
    long long N;
    FastDiv div_nx, div_ny;   // node index -> (x, y, z) for fluid-list kernels
    int ncomp;
    int collision;
    int common_velocity;
    int bc[6];
    int psi_kind[2];
    int eos[2];
    T omega[2];          // 1 / tau
    T rates[2][19];      // MRT rates, stress = 1/tau, conserved = 0
    T rates_n[2][19];    // rates[k][a] / |M_a|^2 (squared norm of moment row a)
    T eos_a[2], eos_b[2], RT[2], alphaT[2], sqrtT[2];
    T alpha_lo[2];                  // hi + lo parts for FP32
    T eos_c[2][5], eos_c_lo[2][5];  // p = rho N(rho) / D(rho): coefficients of N, hi + lo
    T two_over_g[2], two_over_g_lo[2];
    T gm12[2], gm12_lo[2];           // -g_kk / 12, hi + lo
    T alpha[2], A[2], g[2][2];
    T oneA[2], oneA_lo[2];   // 1 - A as hi + lo
    T wet_phi[2], wet_drho[2], rho_min[2], rho_max[2];
    T accel[2][3];
    T rho_ref[2];        // 16-bit population storage holds f_i - w_i rho_ref[k] (0 otherwise)
    T kappa_g2[2];       // kappa g_kk / 2 of the surface-tension source (D2Q9 MRT; 0 = off)
    int forcing_moment;  // 1: moment-space forcing of Eq. mrt_surface (D2Q9), 0: EDM (Eq. edm)
    T bc_rho[2][2];      // [x side][component]
};

// Operations dispatched to the per-(lattice, type) translation units.
enum : int {
    OP_DENSITY = 0,      // rho, psi (U) at fluid nodes from the pre-stream buffer
    OP_VIRTUAL = 1,      // virtual density / psi at boundary solids
    OP_COLLIDE = 2,      // fused gather + force + collision + EDM -> post-collision buffer
    OP_INIT_EQ = 3,      // post-stream populations := f^eq(rho0, u0)
    OP_SET_POPS = 4,     // post-stream populations := given array
    OP_GET_POPS = 5,     // gather post-stream populations into an array
    OP_MACRO = 6,        // rho, u = (j + F/2) / rho into arrays
    OP_DIAG = 7,         // mass / momentum / residual partial sums (deterministic)
    OP_FUSED = 8,        // single-pass step (periodic, no solids, D3Q19)
    OP_STREAM = 9        // free streaming only: gathered populations stored unchanged (bandwidth probe)
};

template <typename T>
struct KArgs {
    Params<T> p;
    const void* f_src;   // pre-stream (post-collision) populations, [K][Q][N] of the storage type
    void* f_dst;         // next pre-stream buffer
    T* psi;              // [K][N]
    T* rho;              // [K][N] (read by the virtual-density pass)
    const uint8_t* solid;
    const int* bsolid;   // boundary-solid node list
    int n_bsolid;
    const int* fluid;    // fluid node list (ascending), or null: kernels run over every node
    int n_fluid;
    const int* fidx;     // with the fluid list: node -> fluid index (-1 at solids), the slot of the
                         // node's populations (fluid-only storage); null: slot = node index
    int geom;            // solids present or a non-periodic face
    int* status;         // device status word
    // operation-specific
    int comp;            // component (-1 = mixture for OP_MACRO)
    const double* in_rho;
    const double* in_u;
    const T* in_f;
    T* out_rho;
    T* out_u;
    T* out_f;
    T* u_prev;           // [D][N] mixture velocity at the last residual request
    int want_residual;
    double* partials;    // [diag_blocks][8]
    double* totals;      // [8]
    int zchunk;          // z planes per CTA of the single-pass step (0 = default)
    int z0, zcount;      // density / collide launches over planes [z0, z0 + zcount) (zcount 0 = all)
    cudaStream_t stream;
};

// One lattice of a batch (lbm_batch_*): its kernel arguments for both buffer
// parities (a[0] pulls from the buffer that holds the current populations) and,
// per batched pass, the first virtual CTA of this lattice in the batch's CTA space.
enum : int { BOP_DENSITY = 0, BOP_VIRTUAL = 1, BOP_COLLIDE = 2 };

template <typename T>
struct BatchItem {
    KArgs<T> a[2];
    long long vb0[3];    // first virtual CTA per pass (density, virtual, collide)
};

// launch shape of one batched pass: CTA size, persistent grid, virtual CTAs in all
struct BatchLaunch {
    int block, grid;
    long long nvb;
};

constexpr int DIAG_BLOCKS = 1024;
constexpr int DIAG_THREADS = 256;

// T: compute type; S: population storage type (T itself, or __half / __nv_bfloat16
// holding shifted values for T = float)
template <class L, typename T, typename S>
cudaError_t run(int op, const KArgs<T>& a);

// One batched pass (BOP_*) over every lattice of the table in one persistent launch.
// The lattices share lattice, types, K, collision and the geometry flag of `shape`.
template <class L, typename T, typename S>
cudaError_t run_batch(int bop, const KArgs<T>& shape, const BatchItem<T>* items, int n_items,
                      const BatchLaunch& launch, int parity, cudaStream_t stream);

}  // namespace lbm
