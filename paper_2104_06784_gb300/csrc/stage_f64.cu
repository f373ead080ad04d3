// stage_f64.cu -- the stage kernels and their launchers for the double element type.
#include "stage_launch.cuh"

namespace moses {

template <>
int launch_stage<double>(const StageArgs<double> &a, int tile, void *stream)
{
    return launch_stage_impl<double>(a, tile, stream);
}

template <>
int launch_stage_rec<double>(const StageArgs<double> &a, void *stream)
{
    return launch_stage_rec_impl<double>(a, stream);
}

template <>
int launch_stage_batch<double>(const StageArgs<double> *args_device, int nsim, const BatchStrip *strips_device, int nstrips,
                            BatchTile *list, unsigned int *list_n, void *stream)
{
    return launch_stage_batch_impl<double>(args_device, nsim, strips_device, nstrips, list, list_n, stream);
}

}  // namespace moses
