// FP32 compute, FP32 shifted fluid populations, bfloat16 solute populations (bulk kernels of two nodes per thread).
#define KTF float
#define KTG __nv_bfloat16
#define KR float
#define KNAME launchers_f32b_n2
#define KPART 2
#include "kernels_impl.cuh"
