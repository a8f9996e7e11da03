// evc_stencil.cu -- matrix-free applies of the periodic finite-difference
// Hamiltonian H = -1/2 Lap_h + V and of the kinetic operator K = -1/2 Lap_h + cI
// on a block of probe columns.  One kernel serves every pass of the
// preconditioned operator C = M (H - sigma I) M (Sec. 2, Eq. negi_T):
//   * the Clenshaw steps of the Chebyshev preconditioner M = p_d(K)
//     (Sec. 6, kinetic-energy preconditioning),
//   * the shifted Hamiltonian (H - sigma_c I) with a per-column shift,
//   * the Jacobi-scaled operator diag(m) (H - sigma I) diag(m),
//   * and the closing term "- beta_i q_{i-1}" of Algorithm 1.
//
// Layout: X[chunk][p][32] with p = x + N*(y + N*z).  Each thread owns one
// 16-byte vector of columns (4 FP32 or 2 FP64 probes) of one (x, y) line and
// marches along z keeping the z-neighbours in a register window; x/y
// neighbours come through L1.  The pass is HBM-bound: it streams the operand
// once and the pointwise operands once.
#include "evc_internal.cuh"

#include <cstring>

namespace evc {
namespace {

template <typename T> struct alignas(16) Pack { T v[16 / sizeof(T)]; };
template <typename T> struct Vec16;
template <> struct Vec16<float> { typedef float4 type; };
template <> struct Vec16<double> { typedef double2 type; };

template <typename T>
__device__ __forceinline__ Pack<T> ldg_pack(const Pack<T>* p)
{
    typename Vec16<T>::type t = __ldg(reinterpret_cast<const typename Vec16<T>::type*>(p));
    Pack<T> r;
    memcpy(&r, &t, 16);
    return r;
}

template <typename T>
__device__ __forceinline__ Pack<T> ld_pack(const Pack<T>* p)
{
    typename Vec16<T>::type t = *reinterpret_cast<const typename Vec16<T>::type*>(p);
    Pack<T> r;
    memcpy(&r, &t, 16);
    return r;
}

template <typename T>
__device__ __forceinline__ void st_pack(Pack<T>* p, const Pack<T>& v)
{
    typename Vec16<T>::type t;
    memcpy(&t, &v, 16);
    *reinterpret_cast<typename Vec16<T>::type*>(p) = t;
}

constexpr int TX = 8;     // points per block along x
constexpr int ZB = 16;    // z planes per block

struct KArgs {
    StencilPass p;
    StencilOp op;
    const int* shift_of;
    const double* sigma;
    const void* jac;
    const int* chunk_active;
    int64_t n;
};

template <typename T, int R, bool JAC>
__global__ void __launch_bounds__(kThreads)
stencil_pass_kernel(KArgs a)
{
    constexpr int W = 16 / sizeof(T);        // columns per thread
    constexpr int LPP = CW / W;              // threads per grid point
    constexpr int TY = kThreads / LPP / TX;  // points per block along y
    const int ch = blockIdx.z;
    if (!a.chunk_active[ch]) return;
    const int N = a.op.N;
    const int lane = threadIdx.x % LPP;
    const int pt = threadIdx.x / LPP;
    const int tilesX = (N + TX - 1) / TX;
    const int x = (blockIdx.x % tilesX) * TX + pt % TX;
    const int y = (blockIdx.x / tilesX) * TY + pt / TX;
    if (x >= N || y >= N) return;            // no block-level barriers below
    const int z0 = blockIdx.y * ZB;
    const int z1 = min(z0 + ZB, N);
    const int64_t n = a.n;

    const Pack<T>* in = reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.in) + ch * a.p.in_cs) + lane;
    const Pack<T>* xv = a.p.x ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.x) + ch * a.p.x_cs) + lane : nullptr;
    const Pack<T>* pv = a.p.prev ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.prev) + ch * a.p.prev_cs) + lane : nullptr;
    const Pack<T>* ppv = a.p.pp ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.pp) + ch * a.p.pp_cs) + lane : nullptr;
    Pack<T>* out = reinterpret_cast<Pack<T>*>(static_cast<T*>(a.p.out) + ch * a.p.out_cs) + lane;
    const T* V = static_cast<const T*>(a.op.V);

    // per-column constants
    const int c0 = ch * CW + lane * W;
    T sig[W], insc[W], a0s[W], ppc[W];
    const T* jr[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int c = c0 + w;
        sig[w] = a.p.useSigma ? (T)a.sigma[c] : (T)0;
        insc[w] = a.p.insc ? (T)a.p.insc[c] : (T)1;
        a0s[w] = (T)(a.p.a0 * (a.p.xs ? a.p.xs[c] : 1.0));
        ppc[w] = a.p.ppc ? (T)a.p.ppc[c] : (T)0;
        jr[w] = JAC ? static_cast<const T*>(a.jac) + (int64_t)a.shift_of[c] * n : nullptr;
    }
    const T k1 = (T)a.p.k1;
    const T c1 = (T)a.op.c1, c2 = (T)a.op.c2;
    const T dg = (T)(a.p.k1 * a.op.cd + a.p.k0);
    const T a2 = (T)a.p.a2;

    // wrapped in-plane neighbour coordinates
    const int xm1 = x == 0 ? N - 1 : x - 1, xp1 = x == N - 1 ? 0 : x + 1;
    const int ym1 = y == 0 ? N - 1 : y - 1, yp1 = y == N - 1 ? 0 : y + 1;
    const int xm2 = (x + N - 2) % N, xp2 = (x + 2) % N;
    const int ym2 = (y + N - 2) % N, yp2 = (y + 2) % N;
    const int64_t NN = (int64_t)N * N;

    auto load = [&](int64_t q) -> Pack<T> {
        Pack<T> v = ldg_pack(in + q * LPP);
        if (JAC) {
#pragma unroll
            for (int w = 0; w < W; ++w) v.v[w] *= __ldg(jr[w] + q);
        }
        return v;
    };

    Pack<T> win[2 * R + 1];
#pragma unroll
    for (int o = -R; o <= R; ++o) {
        const int zz = ((z0 + o) % N + N) % N;
        win[o + R] = load(x + (int64_t)N * y + NN * zz);
    }

    for (int z = z0; z < z1; ++z) {
        const int64_t rowz = NN * z;
        const int64_t p = x + (int64_t)N * y + rowz;
        Pack<T> s1 = load(xm1 + (int64_t)N * y + rowz);
        {
            const Pack<T> t1 = load(xp1 + (int64_t)N * y + rowz);
            const Pack<T> t2 = load(x + (int64_t)N * ym1 + rowz);
            const Pack<T> t3 = load(x + (int64_t)N * yp1 + rowz);
#pragma unroll
            for (int w = 0; w < W; ++w)
                s1.v[w] += t1.v[w] + t2.v[w] + t3.v[w] + win[R - 1].v[w] + win[R + 1].v[w];
        }
        Pack<T> s2;
        if (R == 2) {
            s2 = load(xm2 + (int64_t)N * y + rowz);
            const Pack<T> t1 = load(xp2 + (int64_t)N * y + rowz);
            const Pack<T> t2 = load(x + (int64_t)N * ym2 + rowz);
            const Pack<T> t3 = load(x + (int64_t)N * yp2 + rowz);
#pragma unroll
            for (int w = 0; w < W; ++w)
                s2.v[w] += t1.v[w] + t2.v[w] + t3.v[w] + win[0].v[w] + win[2 * R].v[w];
        }
        const T vp = a.p.useV ? V[p] : (T)0;
        Pack<T> res;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            T off = c1 * s1.v[w];
            if (R == 2) off += c2 * s2.v[w];
            T st = k1 * off + (dg + vp - sig[w]) * win[R].v[w];
            if (JAC) st *= __ldg(jr[w] + p);
            res.v[w] = insc[w] * st;
        }
        if (xv) {
            const Pack<T> t = ld_pack(xv + p * LPP);
#pragma unroll
            for (int w = 0; w < W; ++w) res.v[w] += a0s[w] * t.v[w];
        }
        if (pv) {
            const Pack<T> t = ld_pack(pv + p * LPP);
#pragma unroll
            for (int w = 0; w < W; ++w) res.v[w] -= a2 * t.v[w];
        }
        if (ppv) {
            const Pack<T> t = ld_pack(ppv + p * LPP);
#pragma unroll
            for (int w = 0; w < W; ++w) res.v[w] -= ppc[w] * t.v[w];
        }
        st_pack(out + p * LPP, res);
        if (z + 1 < z1) {
#pragma unroll
            for (int o = 0; o < 2 * R; ++o) win[o] = win[o + 1];
            const int zz = (z + 1 + R) % N;
            win[2 * R] = load(x + (int64_t)N * y + NN * zz);
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_stencil_pass(const StencilOp& op, const Run& r, const StencilPass& p,
                                bool jacobi, cudaStream_t st)
{
    constexpr int W = 16 / sizeof(T);
    constexpr int LPP = CW / W;
    constexpr int TY = kThreads / LPP / TX;
    KArgs a;
    a.p = p;
    a.op = op;
    a.shift_of = r.shift_of;
    a.sigma = r.sigma;
    a.jac = r.jac;
    a.chunk_active = r.chunk_active;
    a.n = r.n;
    const int N = op.N;
    dim3 grid(((N + TX - 1) / TX) * ((N + TY - 1) / TY), (N + ZB - 1) / ZB, r.nchunk);
    if (op.order == 2) {
        if (jacobi) stencil_pass_kernel<T, 1, true><<<grid, kThreads, 0, st>>>(a);
        else stencil_pass_kernel<T, 1, false><<<grid, kThreads, 0, st>>>(a);
    } else {
        if (jacobi) stencil_pass_kernel<T, 2, true><<<grid, kThreads, 0, st>>>(a);
        else stencil_pass_kernel<T, 2, false><<<grid, kThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t launch_stencil_pass<float>(const StencilOp&, const Run&, const StencilPass&,
                                                bool, cudaStream_t);
template cudaError_t launch_stencil_pass<double>(const StencilOp&, const Run&, const StencilPass&,
                                                 bool, cudaStream_t);

}  // namespace evc
