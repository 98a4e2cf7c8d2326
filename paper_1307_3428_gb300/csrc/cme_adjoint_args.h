// Arguments of the adjoint (backward) kernels, shared by the host API and the kernel units.
#pragma once

#include "cme_internal.h"

namespace cme {

struct AdjArgs {
    StepArgs s;              // the group's forward arguments (propagators, twiddles, pump...)
    long long nsteps;        // steps of the forward run
    long long K;             // steps per segment
    long long S;             // segments
    long long total;         // modes in the batch (stride of the per-segment arrays)
    const void* ckpt_hi;     // [S][total] field at the segment starts (transform order)
    const void* ckpt_lo;     // [S][total] compensation words (FP32)
    void* seg;               // [K][total] hi part of the states of the current segment
    void* ybuf;              // [3][total] y1 = F(D), k2, k3 of the step being reversed
    void* dbar;              // [total] in: cotangent of the final field; out: of the initial
    double2* gL;             // [total] accumulated cotangent of L_mu (re: dL/dRe L, im: dL/dIm L)
    double2* pbar;           // [ninst] cotangent of the pump sqrt(kappa_ext) A_in
};

}  // namespace cme
