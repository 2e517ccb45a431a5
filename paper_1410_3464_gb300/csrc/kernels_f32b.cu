// FP32 compute, FP32 shifted fluid populations, bfloat16 solute populations.
#define KTF float
#define KTG __nv_bfloat16
#define KR float
#define KNAME launchers_f32b
#define KPART 1
#include "kernels_impl.cuh"
