"""GB300-native evaluation of LambdaCDM+radiation+curvature distances via
Carlson's symmetric elliptic integrals (Karchev, arXiv:2212.01937).

The compute path is the C-ABI library ``liblcdm`` (CUDA, sm_103a) built from
``csrc/``; ``lcdm`` is its thin Python binding.  Importing this package does
not load the library; the first call into ``lcdm`` does, and raises if it is
missing.
"""
__all__ = ["lcdm", "workloads"]
