// FP32 compute, FP32 shifted fluid populations, IEEE half solute populations.
#define KTF float
#define KTG __half
#define KR float
#define KNAME launchers_f32h
#define KPART 1
#include "kernels_impl.cuh"
