// tls_types.h -- storage formats and sublattice geometry shared by host and device code.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define TLS_HD __host__ __device__
#else
#define TLS_HD
#endif

namespace tls {

enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2, P_BF16 = 3 };

// W storage formats: precision x reals per 3x3 matrix.
enum WFmtId {
    W_F64_18 = 0,
    W_F32_18 = 1,
    W_F32_12 = 2,
    W_F32_8 = 3,
    W_F16_18 = 4,
    W_F16_12 = 5,
    W_BF16_18 = 6,
    W_BF16_12 = 7,
    W_NFMT = 8
};

TLS_HD constexpr int wfmt_bytes(int f)
{
    return f == W_F64_18 ? 144 : f == W_F32_18 ? 72 : f == W_F32_12 ? 48 : f == W_F32_8 ? 32
         : f == W_F16_18 || f == W_BF16_18 ? 36 : 24;
}

// Vector storage: bytes per site and vector.
TLS_HD constexpr int vfmt_bytes(int p)
{
    return p == P_F64 ? 48 : p == P_F32 ? 24 : 16;
}

// Sublattice geometry: half extents, sites per sublattice, plane stride.
struct SubGeom {
    int hx, hy, hz;  // half extents
    int Vs;          // hx * hy * hz
    int64_t Ps;      // plane stride (Vs rounded up to 32)
};

// Device error word bits.
enum DevErr {
    DERR_BOUNDS = 1,      // an index check failed (checked builds)
    DERR_TIMEOUT = 2,     // a bounded barrier ran out of polls
    DERR_RECON8 = 4,      // 8-real form met |W00| ~ 1
    DERR_PROJECT = 8,     // a link projection onto SU(3) met a singular matrix or did not settle
};

}  // namespace tls
