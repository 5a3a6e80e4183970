// Runtime-degree ("wide") neighbour records and their coupling sums, shared by
// the runtime-degree sweep kernels of the plain contexts (pt2d_generic.cu) and
// the runtime-degree path of the batched kernel (pt2d_batch.cu).
//
// Record of one position, in ints, padded to whole int4s:
//   [nb x DC | lk x DL | pid | 2h | pad to even | (lo, hi) x DC/4 | K x DL | k]
// DC is the coupling degree rounded up to a multiple of 4 (padding neighbours
// point at the slab's zero row with J = 0); the spin id sits at DC + DL as in
// every record layout of the library.  Couplings are packed four at a time as
// two words of bytes, J = 256 hi + lo with lo = J & 0xff (unsigned) and
// hi = J >> 8 (signed), so that sum_k J_k s_k over four couplings is two
// four-way byte dot products (dp4a) per walker: exact integer arithmetic, the
// same sums as one multiply-add per coupling.  K x DL and k (penalty terms)
// are present only when the instance has them.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace pt2d {

// Int offset of the packed couplings in a wide record.
__host__ __device__ __forceinline__ int wide_jpack_offset(int DC, int DL) { return (DC + DL + 3) & ~1; }

// Ints of a wide record before padding to int4s.
__host__ __device__ __forceinline__ int wide_record_ints(int DC, int DL, bool penalty) {
    return wide_jpack_offset(DC, DL) + DC / 2 + (penalty ? DL + 1 : 0);
}

#ifdef __CUDACC__
// sum_i a.byte_i (signed) * b.byte_i (unsigned) + c
__device__ __forceinline__ int dp4a_su(uint32_t a, uint32_t b, int c) {
    int d;
    asm("dp4a.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// sum_i a.byte_i (signed) * b.byte_i (signed) + c
__device__ __forceinline__ int dp4a_ss(uint32_t a, uint32_t b, int c) {
    int d;
    asm("dp4a.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Byte transpose of four spin words (word k = the quad's four walkers at
// neighbour k): w_b = the four neighbours' spins of walker b.
__device__ __forceinline__ void transpose4(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3, uint32_t &w0,
                                           uint32_t &w1, uint32_t &w2, uint32_t &w3) {
    uint32_t t0, t1, t2, t3;
    asm("prmt.b32 %0, %1, %2, 0x5140;" : "=r"(t0) : "r"(x0), "r"(x1));
    asm("prmt.b32 %0, %1, %2, 0x7362;" : "=r"(t1) : "r"(x0), "r"(x1));
    asm("prmt.b32 %0, %1, %2, 0x5140;" : "=r"(t2) : "r"(x2), "r"(x3));
    asm("prmt.b32 %0, %1, %2, 0x7362;" : "=r"(t3) : "r"(x2), "r"(x3));
    asm("prmt.b32 %0, %1, %2, 0x5410;" : "=r"(w0) : "r"(t0), "r"(t2));
    asm("prmt.b32 %0, %1, %2, 0x7632;" : "=r"(w1) : "r"(t0), "r"(t2));
    asm("prmt.b32 %0, %1, %2, 0x5410;" : "=r"(w2) : "r"(t1), "r"(t3));
    asm("prmt.b32 %0, %1, %2, 0x7632;" : "=r"(w3) : "r"(t1), "r"(t3));
}

// sum_k J_k s_k for the quad's four walkers over the record's DC couplings.
// rc: the record (global memory, read through the read-only path); fetch(ref)
// returns the quad's spin word at a neighbour reference.  LEAN folds the high
// bytes' dot product into the running sum at once (one more multiply-add per
// walker and group, four fewer live registers: for kernels at their register
// cap, where the separate sums spill).
template <bool LEAN, typename Fetch>
__device__ __forceinline__ void wide_coupling_sums(const int *rc, int DC, int jo, Fetch fetch, int &c0, int &c1,
                                                   int &c2, int &c3) {
    int u0 = 0, u1 = 0, u2 = 0, u3 = 0, v0 = 0, v1 = 0, v2 = 0, v3 = 0;
    const int4 *nb = reinterpret_cast<const int4 *>(rc);
    const int2 *jp = reinterpret_cast<const int2 *>(rc + jo);
    for (int g = 0; g < DC / 4; ++g) {
        const int4 r = __ldg(nb + g);
        const int2 j = __ldg(jp + g);
        uint32_t w0, w1, w2, w3;
        transpose4(fetch(r.x), fetch(r.y), fetch(r.z), fetch(r.w), w0, w1, w2, w3);
        const uint32_t lo = static_cast<uint32_t>(j.x), hi = static_cast<uint32_t>(j.y);
        if (LEAN) {
            u0 = dp4a_su(w0, lo, u0 + 256 * dp4a_ss(w0, hi, 0));
            u1 = dp4a_su(w1, lo, u1 + 256 * dp4a_ss(w1, hi, 0));
            u2 = dp4a_su(w2, lo, u2 + 256 * dp4a_ss(w2, hi, 0));
            u3 = dp4a_su(w3, lo, u3 + 256 * dp4a_ss(w3, hi, 0));
        } else {
            u0 = dp4a_su(w0, lo, u0);
            u1 = dp4a_su(w1, lo, u1);
            u2 = dp4a_su(w2, lo, u2);
            u3 = dp4a_su(w3, lo, u3);
            v0 = dp4a_ss(w0, hi, v0);
            v1 = dp4a_ss(w1, hi, v1);
            v2 = dp4a_ss(w2, hi, v2);
            v3 = dp4a_ss(w3, hi, v3);
        }
    }
    c0 = u0 + 256 * v0;
    c1 = u1 + 256 * v1;
    c2 = u2 + 256 * v2;
    c3 = u3 + 256 * v3;
}
#endif

}  // namespace pt2d
