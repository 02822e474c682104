// window_coop.cu -- instantiations of the cooperative window kernel for one
// histogram form (PIC_WINDOW_HIST: 0, 1 or 2) and fine solver
// (PIC_WINDOW_SOLVER: 0 classical RK4, 1 Lawson RK4), with both mesh
// locates and both load paths.  The build compiles this file once per pair,
// in parallel, and window.cu reaches the kernels through the exported table.
#include "pic_internal.h"
#include "window_common.cuh"
#include "window_coop.cuh"

#if !defined(PIC_WINDOW_HIST) || !defined(PIC_WINDOW_SOLVER)
#error "define PIC_WINDOW_HIST and PIC_WINDOW_SOLVER"
#endif

#define PIC_CAT4(a, b, c, d) a##b##c##d
#define PIC_KERNEL_TABLE(h, s) PIC_CAT4(window_coop_kernel_h, h, _s, s)

namespace pic {

void* PIC_KERNEL_TABLE(PIC_WINDOW_HIST, PIC_WINDOW_SOLVER)(int pow2, int stage) {
    constexpr int H = PIC_WINDOW_HIST, S = PIC_WINDOW_SOLVER;
    if (pow2) return stage ? (void*)k_window_coop<S, H, 1, 1> : (void*)k_window_coop<S, H, 1, 0>;
    return stage ? (void*)k_window_coop<S, H, 0, 1> : (void*)k_window_coop<S, H, 0, 0>;
}

}  // namespace pic
