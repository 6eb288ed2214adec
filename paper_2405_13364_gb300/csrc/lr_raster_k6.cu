// Rasteriser instantiation for a per-pixel sorter of capacity K = 6.
#include "lr_raster.cuh"
LR_DEFINE_RASTER(6)
