"""GB300 (sm_103a) mixed precision Gram-matrix thin SVD -- Python binding.

Placeholder: the binding is written together with the CUDA library.
"""
