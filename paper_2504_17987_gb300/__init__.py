"""GB300 (sm_103a) implementation of the correction hot path of RapidPIV
(arXiv 2504.17987): image deformation by a predictor, zero-normalised
correlation over a +-r search, integer peak, three-point Gaussian fit,
universal outlier detection with median replacement and vorticity, with a
coarse-to-fine correlation pyramid standing in for the optical-flow engine.

The compute runs in librpiv.so (CUDA kernels behind a C ABI, include/rpiv.h);
this package is its binding plus the serving loop."""
from .binding import (Config, CorrelationScore, Engine, RpivError, decode_info, load, refine, stage_correlate,
                      stage_downsample, stage_ema, stage_interp, stage_preprocess, stage_status, stage_validate,
                      stage_vorticity, to_device, validate_config)

__all__ = ["Config", "CorrelationScore", "Engine", "RpivError", "decode_info", "load", "refine", "stage_correlate",
           "stage_downsample", "stage_ema", "stage_interp", "stage_preprocess", "stage_status", "stage_validate",
           "stage_vorticity", "to_device", "validate_config"]
