// FP32 compute, FP32 shifted fluid populations, IEEE half solute populations (bulk kernels of two nodes per thread).
#define KTF float
#define KTG __half
#define KR float
#define KNAME launchers_f32h_n2
#define KPART 2
#include "kernels_impl.cuh"
