// mhd_fp32.cu -- step pipelines instantiated for one precision (float,float,float).
#include "mhd_engine.cuh"

mhd_step_fn mhd_pick_fp32(int integ, int recon, int solver, cudaError_t* attr)
{
    return mhd::pick_step<float,float,float>(integ, recon, solver, attr);
}
