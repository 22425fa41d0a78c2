"""GB300-native complex constrained TV denoising and TV-regularised phase
retrieval (Gao & Cao, arXiv 2109.05496).

The compute path is ``libctv.so`` (hand-written CUDA for sm_103a, C ABI in
``include/ctv.h``); this package marshals torch tensors into it. Importing the
package does not load the library; the first call does, and fails loudly if it
has not been built.
"""
from .api import (TV_TYPES, Constraint, NO_CONSTRAINT, configs, ctv_denoise, ctv_denoise_batched,  # noqa: F401
                  denoise, get_last_error, make_opts, workspace, PRPlan, Plan, ctv_prox_grad_step,
                  UnrolledFGP, denoise_unrolled)

__all__ = ["TV_TYPES", "Constraint", "NO_CONSTRAINT", "configs", "ctv_denoise", "ctv_denoise_batched",
           "denoise", "get_last_error", "make_opts", "workspace", "PRPlan", "Plan", "ctv_prox_grad_step",
           "UnrolledFGP", "denoise_unrolled"]
