// Discrete decisions of one pixel in one sweep, recorded by the sweep kernel (a
// byte per pixel) so that the adjoint differentiates the branch the forward took.
#pragma once

namespace pv {
constexpr unsigned char BR_VALID = 0x1;  // the photometric factor was active
constexpr unsigned char BR_HUBER = 0x2;  // its Huber weight was below 1
constexpr unsigned char BR_SKIP = 0x4;   // the belief solve failed and tau was set to 0
}  // namespace pv
