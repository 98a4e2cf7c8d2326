// Arguments of the adjoint (backward) kernels, shared by the host API and the kernel units.
#pragma once

#include "cme_internal.h"

namespace cme {

struct AdjArgs {
    StepArgs s;              // the group's forward arguments (propagators, twiddles, pump...)
    long long nsteps;        // steps of the forward run
    long long K;             // steps per segment
    long long S;             // segments
    long long seg;           // the segment this launch handles
    long long total;         // modes in the batch (stride of the per-segment arrays)
    const void* ckpt_hi;     // [S][total] field at the segment starts (transform order)
    const void* ckpt_lo;     // [S][total] compensation words (FP32)
    void* stages;            // [slots][K][ADJ_VECS][total]: per step of a segment, D,
                             // y1 = F(D), k2, k3, then a = IDFT(stage input) of D, x2, x3, x4
                             // (RK4IP), or D, the time-domain field a of the Kerr flow and the
                             // state after it (Strang); segment seg uses slot `slot`
    void* dbar;              // [total] cotangent of the field (carried between launches)
    double2* gL;             // [total] accumulated cotangent of L_mu (re: dL/dRe L, im: dL/dIm L)
    double2* pbar;           // [ninst] cotangent of the pump sqrt(kappa_ext) A_in (RK4IP),
                             // of the pump increment c of the linear half flows (Strang)
    int method;              // METHOD_RK4IP or METHOD_STRANG
    long long slot;          // slot of A.stages holding segment seg's per-step data
    long long ckpt_slot;     // checkpoint the recomputation starts from
    void* out_hi;            // recomputation: where its final state goes (null: nowhere)
    void* out_lo;
};

// Kernel roles of one segment: recompute the states and stage values, or run it backwards.
enum { ADJ_BACKWARD = 0, ADJ_RECOMPUTE = 1 };
// Field vectors stored per step of a segment.
constexpr int ADJ_VECS = 8;

}  // namespace cme
