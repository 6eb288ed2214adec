// Rasteriser instantiation with per-strip shared set-up for a per-pixel sorter of capacity K = 2.
#include "lr_raster_strip.cuh"
LR_DEFINE_RASTER_STRIP(2)
