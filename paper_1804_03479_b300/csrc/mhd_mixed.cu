// mhd_mixed.cu -- step pipelines instantiated for one precision (float,float,double).
#include "mhd_engine.cuh"

mhd_step_fn mhd_pick_mixed(int integ, int recon, int solver, cudaError_t* attr)
{
    return mhd::pick_step<float,float,double>(integ, recon, solver, attr);
}
