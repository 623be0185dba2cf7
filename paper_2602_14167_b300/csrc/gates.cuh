// Gate matrices on the device, FP64 (shared by the matrix prologue and the
// state-pass adjoint).  Conventions: R_P(t) = exp(-i t P / 2); a k-qubit
// gate's local index is sum_j bit(q[j]) << (k-1-j) (q[0] most significant);
// CX(control, target); CP(phi) = diag(1, 1, 1, e^{i phi}); RP's Pauli word
// is the op's pool_off field (digit j, 2 bits: 0 I, 1 X, 2 Y, 3 Z, on q[j]).
#pragma once

#include <cuda_runtime.h>

#include "internal.hpp"

namespace tcng {

// Matrix of one gate in its own local order (q[0] most significant).
__device__ inline void gate_matrix_d(const BuildOp& op, double ang, double2* M, int d,
                              const double2* pool) {
    for (int i = 0; i < d * d; ++i) M[i] = make_double2(0, 0);
    double c, s;
    const double r2 = 0.70710678118654752440;
    switch (op.code) {
    case TCNG_I: M[0].x = 1; M[3].x = 1; break;
    case TCNG_X: M[1].x = 1; M[2].x = 1; break;
    case TCNG_Y: M[1].y = -1; M[2].y = 1; break;
    case TCNG_Z: M[0].x = 1; M[3].x = -1; break;
    case TCNG_H: M[0].x = r2; M[1].x = r2; M[2].x = r2; M[3].x = -r2; break;
    case TCNG_S: M[0].x = 1; M[3].y = 1; break;
    case TCNG_T: M[0].x = 1; M[3] = make_double2(r2, r2); break;
    case TCNG_RX:
        sincos(0.5 * ang, &s, &c);
        M[0].x = c; M[1].y = -s; M[2].y = -s; M[3].x = c; break;
    case TCNG_RY:
        sincos(0.5 * ang, &s, &c);
        M[0].x = c; M[1].x = -s; M[2].x = s; M[3].x = c; break;
    case TCNG_RZ:
        sincos(0.5 * ang, &s, &c);
        M[0] = make_double2(c, -s); M[3] = make_double2(c, s); break;
    case TCNG_CX: M[0].x = 1; M[5].x = 1; M[11].x = 1; M[14].x = 1; break;
    case TCNG_CZ: M[0].x = 1; M[5].x = 1; M[10].x = 1; M[15].x = -1; break;
    case TCNG_CP:
        sincos(ang, &s, &c);
        M[0].x = 1; M[5].x = 1; M[10].x = 1; M[15] = make_double2(c, s); break;
    case TCNG_SWAP: M[0].x = 1; M[6].x = 1; M[9].x = 1; M[15].x = 1; break;
    case TCNG_RZZ:
        sincos(0.5 * ang, &s, &c);
        M[0] = make_double2(c, -s); M[5] = make_double2(c, s);
        M[10] = make_double2(c, s); M[15] = make_double2(c, -s); break;
    case TCNG_RP: {   // cos(t/2) I - i sin(t/2) P, P = (x)_j sigma_{w_j}; pool_off holds the word
        sincos(0.5 * ang, &s, &c);
        const int k = op.k;
        for (int r = 0; r < d; ++r)
            for (int col = 0; col < d; ++col) {
                double pr = 1.0, pi = 0.0;   // product of the factors' entries
                for (int j = 0; j < k && (pr != 0.0 || pi != 0.0); ++j) {
                    const int w = (int)((op.pool_off >> (2 * j)) & 3);
                    const int a = (r >> (k - 1 - j)) & 1, b = (col >> (k - 1 - j)) & 1;
                    double er = 0.0, ei = 0.0;   // sigma_w[a][b]
                    if (w == 0) er = a == b ? 1.0 : 0.0;
                    else if (w == 1) er = a != b ? 1.0 : 0.0;
                    else if (w == 2) ei = a == b ? 0.0 : (a ? 1.0 : -1.0);
                    else er = a == b ? (a ? -1.0 : 1.0) : 0.0;
                    const double nr = pr * er - pi * ei, ni = pr * ei + pi * er;
                    pr = nr;
                    pi = ni;
                }
                // -i s P + c I
                M[r * d + col] = make_double2((r == col ? c : 0.0) + s * pi, -s * pr);
            }
        break;
    }
    default:  // U1 / U2 / UK
        for (int i = 0; i < d * d; ++i) M[i] = pool[op.pool_off + i];
        break;
    }
}

}  // namespace tcng
