// Tape recording and reverse-mode gradients (placeholder until the adjoint kernels land).
#include "mpm_ctx.cuh"

struct mpm_tape {};

int mpm_tape_record_substep(mpm_ctx*, float) { return MPM_ERR_STATE; }
void mpm_tape_free(mpm_ctx* c) { if (c && c->tape) { delete c->tape; c->tape = nullptr; } }
extern "C" int mpm_tape_begin(mpm_ctx*) { return MPM_ERR_STATE; }
extern "C" int mpm_backward(mpm_ctx*, const float*, const float*, float*, float*, float*, int) { return MPM_ERR_STATE; }
