// evc_csr.cu -- the preconditioned shifted operator for a CSR matrix,
//   w = M (A - sigma_c I) M q_i - beta_i q_{i-1}       (Algorithm 1, first
// line of the loop body), with M = I or the Jacobi scaling
// M = diag((|a_rr - sigma| + eps)^(-1/2)) fused as row and column scales;
// or, for the T^{-1}-inner-product process (Sec. 4, Eq. lanT1) with T = M^2,
//   w = T (A - sigma_c I) y_i - beta_i y_{i-1},
// where T is a row scale only and the gathered rows are not scaled.
//
// Row r of C x is  m_r sum_{j != r} a_rj m_j x_j  +  d_r x_r  with the
// diagonal d_r = (a_rr - sigma) m_r^2 (or a_rr - sigma without M) taken from
// a per-shift array formed in FP64: the stored diagonal entries are skipped in
// the row sum, so in FP32 the shift never cancels against a_rr, and a rounded
// a_rr never reaches m_r^2, which magnifies it by up to 1/eps.
//
// Every gathered x row of a chunk is one contiguous 128-byte (FP32) / 256-byte
// (FP64) segment; q_i = s_i P_i is scaled on the fly.
#include "evc_internal.cuh"

#include <cstring>
#include <type_traits>

namespace evc {
namespace {

struct CArgs {
    CsrOp op;
    const void* x;          // slot i-1 of the basis (P_i)
    const void* pp;         // slot i-2 (P_{i-1}) or null
    void* out;              // slot i
    int64_t chunk_stride;
    const double* insc;     // s_i per column
    const double* ppc;      // beta_i s_{i-1} per column
    const int* shift_of;
    const void* jac;
    const void* dsh;        // T[S][n] diagonal of the shifted (scaled) operator
    const int* chunk_active;
};

template <typename T> struct alignas(16) Pack { T v[16 / sizeof(T)]; };
template <typename T> struct Vec16;
template <> struct Vec16<float> { typedef float4 type; };
template <> struct Vec16<double> { typedef double2 type; };

// Row sums are accumulated entry by entry, acc = fma(a_rj, x_j m_j, acc), with
// the product and the fused multiply-add rounded explicitly, so that every
// specialisation of the pass (uniform-shift chunks or not, any block size)
// gives bitwise the same rows: a column's result must not depend on which
// kernel its batch ran.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ Pack<T> ldg16(const T* p)
{
    typename Vec16<T>::type t = __ldg(reinterpret_cast<const typename Vec16<T>::type*>(p));
    Pack<T> r;
    memcpy(&r, &t, 16);
    return r;
}

// A group of LPR = CW / W lanes owns one row of one chunk; each lane holds W
// consecutive columns (one 16-byte vector), so one gather instruction of the
// warp fetches 32/LPR whole x rows.  Rows are visited in the order of
// op.perm (rows sorted by length, longest first) so the rows sharing a warp
// have similar lengths; each group broadcasts the row's (col, val) pairs from
// its own lanes with warp shuffles.  UNI: every chunk's 32 columns belong to
// one shift (m a multiple of 32, or one shift), so a gathered entry needs one
// Jacobi scale, not one per column.  PM: PM_NONE, PM_JACOBI (row and column
// scales m) or PM_TLEFT (row scale T = m^2 only; jac then holds m^2).
template <typename T, int PM, bool UNI, int NT>
__global__ void __launch_bounds__(NT)
csr_pass_kernel(CArgs a)
{
    constexpr bool JAC = PM == PM_JACOBI;       // gathered rows scaled by m
    constexpr bool ROWS = PM != PM_NONE;        // output rows scaled
    constexpr int W = 16 / sizeof(T);
    constexpr int LPR = CW / W;                 // lanes per row
    constexpr int RPW = 32 / LPR;               // rows per warp
    const int ch = blockIdx.y;
    if (!a.chunk_active[ch]) return;
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPR, sub = lane % LPR;
    const int64_t slotrow = ((int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5)) * RPW + grp;
    const int64_t n = a.op.n;
    const bool valid = slotrow < n;
    const int64_t row = valid ? (a.op.perm ? (int64_t)a.op.perm[slotrow] : slotrow) : 0;
    const int c0 = ch * CW + sub * W;
    const T* x = static_cast<const T*>(a.x) + ch * a.chunk_stride;
    const T* val = static_cast<const T*>(a.op.val);
    constexpr int NJ = UNI ? 1 : W;             // Jacobi scale arrays in use
    const T* jr[NJ];
#pragma unroll
    for (int w = 0; w < NJ; ++w)
        jr[w] = ROWS ? static_cast<const T*>(a.jac) + (int64_t)a.shift_of[c0 + w] * n : nullptr;

    const int64_t beg = valid ? a.op.row_ptr[row] : 0, end = valid ? a.op.row_ptr[row + 1] : 0;
    // the warp walks the longest of its rows; shorter rows contribute zeros
    int64_t len = end - beg, mx = len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, (int64_t)__shfl_xor_sync(0xffffffffu, mx, o));
    T acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = 0;
    for (int64_t k0 = 0; k0 < mx; k0 += LPR) {
        const int64_t kk = beg + k0 + sub;
        int mycol = (int)row;
        T myval = 0;
        if (k0 + sub < len) {
            mycol = __ldg(a.op.col + kk);
            myval = mycol == (int)row ? (T)0 : __ldg(val + kk);   // diagonal: from dsh
        }
        const int cnt = (int)min((int64_t)LPR, mx - k0);
        int t = 0;
        for (; t + 1 < cnt; t += 2) {
            const int ca = __shfl_sync(0xffffffffu, mycol, grp * LPR + t);
            const int cb = __shfl_sync(0xffffffffu, mycol, grp * LPR + t + 1);
            const T va = __shfl_sync(0xffffffffu, myval, grp * LPR + t);
            const T vb = __shfl_sync(0xffffffffu, myval, grp * LPR + t + 1);
            Pack<T> xa = ldg16(x + (int64_t)ca * CW + sub * W);
            Pack<T> xb = ldg16(x + (int64_t)cb * CW + sub * W);
            T ma = 1, mb = 1;
            if (JAC && UNI) { ma = __ldg(jr[0] + ca); mb = __ldg(jr[0] + cb); }
#pragma unroll
            for (int w = 0; w < W; ++w) {
                T sa = xa.v[w], sb = xb.v[w];
                if (JAC && UNI) { sa = mul_rn(sa, ma); sb = mul_rn(sb, mb); }
                if (JAC && !UNI) {
                    sa = mul_rn(sa, __ldg(jr[w] + ca));
                    sb = mul_rn(sb, __ldg(jr[w] + cb));
                }
                acc[w] = fma_rn(vb, sb, fma_rn(va, sa, acc[w]));
            }
        }
        if (t < cnt) {
            const int ca = __shfl_sync(0xffffffffu, mycol, grp * LPR + t);
            const T va = __shfl_sync(0xffffffffu, myval, grp * LPR + t);
            Pack<T> xa = ldg16(x + (int64_t)ca * CW + sub * W);
            const T ma = JAC && UNI ? __ldg(jr[0] + ca) : (T)1;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                T sa = xa.v[w];
                if (JAC && UNI) sa = mul_rn(sa, ma);
                if (JAC && !UNI) sa = mul_rn(sa, __ldg(jr[w] + ca));
                acc[w] = fma_rn(va, sa, acc[w]);
            }
        }
    }
    if (!valid) return;
    const Pack<T> cen = ldg16(x + row * CW + sub * W);
    const T* pp = a.pp ? static_cast<const T*>(a.pp) + ch * a.chunk_stride : nullptr;
    Pack<T> prev;
    if (pp) prev = ldg16(pp + row * CW + sub * W);
    const T* dsh = static_cast<const T*>(a.dsh);
    Pack<T> res;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int c = c0 + w;
        T r = acc[w];
        if (ROWS) r = mul_rn(r, __ldg(jr[UNI ? 0 : w] + row));
        r = fma_rn(__ldg(dsh + (int64_t)a.shift_of[c] * n + row), cen.v[w], r);
        r = mul_rn(r, (T)a.insc[c]);
        if (pp) r = fma_rn(-(T)a.ppc[c], prev.v[w], r);
        res.v[w] = r;
    }
    typename Vec16<T>::type o;
    memcpy(&o, &res, 16);
    *reinterpret_cast<typename Vec16<T>::type*>(static_cast<T*>(a.out) + ch * a.chunk_stride +
                                                  row * CW + sub * W) = o;
}

}  // namespace

template <typename T>
cudaError_t launch_csr_pass(const CsrOp& op, const Run& r, int i, int pmode, cudaStream_t st)
{
    // step i reads slot i-1 (q_i), slot i-2 (q_{i-1}) and writes slot i
    CArgs a;
    a.op = op;
    T* basis = static_cast<T*>(r.basis);
    a.x = basis + (int64_t)(i - 1) * r.slot_stride;
    // the three-term term -beta_i q_{i-1} is Lanczos only
    a.pp = (i >= 2 && !r.arnoldi) ? basis + (int64_t)(i - 2) * r.slot_stride : nullptr;
    a.out = basis + (int64_t)i * r.slot_stride;
    a.chunk_stride = r.chunk_stride;
    a.insc = r.scl + (int64_t)(i - 1) * r.ncol;
    a.ppc = r.ppc;
    a.shift_of = r.shift_of;
    a.jac = r.jac;
    a.dsh = r.dsh;
    a.chunk_active = r.chunk_active;
    constexpr int RPW = 32 / (CW / (16 / (int)sizeof(T)));
    const int nt = op.threads > 0 ? op.threads : kThreads;
    const int rows_per_block = (nt / 32) * RPW;
    dim3 grid((unsigned)((op.n + rows_per_block - 1) / rows_per_block), r.nchunk);
    // every chunk's columns share one shift when m is a multiple of 32 (the
    // padding columns of the last chunk take the last shift) or S = 1
    const bool uni = r.S == 1 || r.m % CW == 0;
    auto go = [&](auto pm_t, auto uni_t, auto nt_t) {
        csr_pass_kernel<T, decltype(pm_t)::value, decltype(uni_t)::value, decltype(nt_t)::value>
            <<<grid, decltype(nt_t)::value, 0, st>>>(a);
    };
    using F = std::false_type;
    using Tr = std::true_type;
    auto by_nt = [&](auto pm_t, auto uni_t) -> bool {
        switch (nt) {
        case 128: go(pm_t, uni_t, std::integral_constant<int, 128>()); return true;
        case 256: go(pm_t, uni_t, std::integral_constant<int, 256>()); return true;
        case 512: go(pm_t, uni_t, std::integral_constant<int, 512>()); return true;
        default: return false;
        }
    };
    using PNone = std::integral_constant<int, PM_NONE>;
    using PJac = std::integral_constant<int, PM_JACOBI>;
    using PTl = std::integral_constant<int, PM_TLEFT>;
    bool ok;
    if (pmode == PM_NONE) ok = by_nt(PNone(), F());
    else if (pmode == PM_JACOBI) ok = uni ? by_nt(PJac(), Tr()) : by_nt(PJac(), F());
    else if (pmode == PM_TLEFT) ok = uni ? by_nt(PTl(), Tr()) : by_nt(PTl(), F());
    else ok = false;
    if (!ok) return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template cudaError_t launch_csr_pass<float>(const CsrOp&, const Run&, int, int, cudaStream_t);
template cudaError_t launch_csr_pass<double>(const CsrOp&, const Run&, int, int, cudaStream_t);

}  // namespace evc
