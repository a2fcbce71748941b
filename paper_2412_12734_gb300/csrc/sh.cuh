// Real spherical-harmonics basis up to degree 3 (the view-dependent colour of
// Sec. 4.2) and its gradient, shared by the preprocess kernels and the
// per-texel SH passes.
#pragma once

#include "gbill_internal.cuh"

namespace gbill {

// ------------------------------------------------------------- SH colour --
// Real SH basis up to degree 3 with the (-1)^m sign: polynomials in the unit
// direction.  Normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times
// sqrt(2) for m != 0) multiplied out with the Legendre coefficients.
constexpr float kY0 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kY2a = 1.09254843059207907f;  // sqrt(15 / pi) / 2
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5 / pi) / 4
constexpr float kY2c = 0.54627421529603959f;  // sqrt(15 / pi) / 4
constexpr float kY3a = 0.59004358992664352f;  // sqrt(35 / (2 pi)) / 4
constexpr float kY3b = 2.89061144264055405f;  // sqrt(105 / pi) / 2
constexpr float kY3c = 0.45704579946446572f;  // sqrt(21 / (2 pi)) / 4
constexpr float kY3d = 0.37317633259011546f;  // sqrt(7 / pi) / 4
constexpr float kY3e = 1.44530572132027738f;  // sqrt(105 / pi) / 4

__device__ __forceinline__ void sh_basis(int D, float x, float y, float z, float Y[16]) {
    Y[0] = kY0;
    if (D < 1) return;
    Y[1] = -kY1 * y;
    Y[2] = kY1 * z;
    Y[3] = -kY1 * x;
    if (D < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kY2a * x * y;
    Y[5] = -kY2a * y * z;
    Y[6] = kY2b * (2.0f * zz - xx - yy);
    Y[7] = -kY2a * x * z;
    Y[8] = kY2c * (xx - yy);
    if (D < 3) return;
    Y[9] = -kY3a * y * (3.0f * xx - yy);
    Y[10] = kY3b * x * y * z;
    Y[11] = -kY3c * y * (4.0f * zz - xx - yy);
    Y[12] = kY3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -kY3c * x * (4.0f * zz - xx - yy);
    Y[14] = kY3e * z * (xx - yy);
    Y[15] = -kY3a * x * (xx - 3.0f * yy);
}

// Gradient of each basis polynomial with respect to (x, y, z).
__device__ __forceinline__ void sh_basis_grad(int D, float x, float y, float z, float G[16][3]) {
    for (int i = 0; i < 16; ++i) G[i][0] = G[i][1] = G[i][2] = 0.0f;
    if (D < 1) return;
    G[1][1] = -kY1;
    G[2][2] = kY1;
    G[3][0] = -kY1;
    if (D < 2) return;
    G[4][0] = kY2a * y; G[4][1] = kY2a * x;
    G[5][1] = -kY2a * z; G[5][2] = -kY2a * y;
    G[6][0] = -2.0f * kY2b * x; G[6][1] = -2.0f * kY2b * y; G[6][2] = 4.0f * kY2b * z;
    G[7][0] = -kY2a * z; G[7][2] = -kY2a * x;
    G[8][0] = 2.0f * kY2c * x; G[8][1] = -2.0f * kY2c * y;
    if (D < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    G[9][0] = -kY3a * 6.0f * x * y; G[9][1] = -kY3a * (3.0f * xx - 3.0f * yy);
    G[10][0] = kY3b * y * z; G[10][1] = kY3b * x * z; G[10][2] = kY3b * x * y;
    G[11][0] = kY3c * 2.0f * x * y; G[11][1] = -kY3c * (4.0f * zz - xx - 3.0f * yy);
    G[11][2] = -kY3c * 8.0f * y * z;
    G[12][0] = -kY3d * 6.0f * x * z; G[12][1] = -kY3d * 6.0f * y * z;
    G[12][2] = kY3d * (6.0f * zz - 3.0f * xx - 3.0f * yy);
    G[13][0] = -kY3c * (4.0f * zz - 3.0f * xx - yy); G[13][1] = kY3c * 2.0f * x * y;
    G[13][2] = -kY3c * 8.0f * x * z;
    G[14][0] = kY3e * 2.0f * x * z; G[14][1] = -kY3e * 2.0f * y * z; G[14][2] = kY3e * (xx - yy);
    G[15][0] = -kY3a * (3.0f * xx - 3.0f * yy); G[15][1] = kY3a * 6.0f * x * y;
}

}  // namespace gbill
