// Host build of the oriented-box fit and test that the closest-point search
// uses (obb.cuh), exported with C linkage for the CPU tests.
#include <string.h>

#include "../paper_2007_07627_gb300/csrc/obb.cuh"

extern "C" {

// pts: cnt float4 (x, y, z, unused); out: 16 floats.
void h_obb_fit(const float *pts, int cnt, float *out) {
    float4 p[64];
    memcpy(p, pts, sizeof(float4) * (size_t)cnt);
    float4 box[4];
    fricp::obb_fit(p, cnt, box);
    memcpy(out, box, sizeof(box));
}

// box: 16 floats from h_obb_fit; xh, xl: 3 floats each.
float h_obb_d2(const float *box, const float *xh, const float *xl) {
    float4 b[4];
    memcpy(b, box, sizeof(b));
    return fricp::obb_eval(b[0], b[1], b[2], b[3], xh, xl);
}

}
