// FP32 compute, FP32 shifted storage of all populations.
#define KTF float
#define KTG float
#define KR float
#define KNAME launchers_f32
#define KPART 1
#include "kernels_impl.cuh"
