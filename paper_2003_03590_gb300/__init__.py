"""GB300-native Gross-Pitaevskii split-step library (hand-written sm_103a CUDA behind a C ABI).

The compute path lives in libgpqt.so (built by ``paper_2003_03590_gb300.build``);
this package only marshals arguments to it.  There is no CPU fallback: importing
``gpqt`` without the built library raises.
"""
from .gpqt import (GP_FLOW_ABC, GP_FLOW_NONE, GP_FLOW_TG, GP_FP32, GP_FP64, GP_SPLIT_KNK, GP_SPLIT_NKN, SUPPORTED_N,
                   GPError, GPEvolve, IncompressibleKineticEnergy, Plan, field_params)

__all__ = ["Plan", "field_params", "GPEvolve", "IncompressibleKineticEnergy", "GPError", "GP_FP32", "GP_FP64",
           "GP_SPLIT_NKN", "GP_SPLIT_KNK", "SUPPORTED_N", "GP_FLOW_NONE", "GP_FLOW_TG", "GP_FLOW_ABC"]
