"""GB300-native small-scale P_l(k) and B_l(k1,k2) estimators (arXiv:2005.01739).

The compute path is the C-ABI library built from ``csrc/`` (CUDA for sm_103a);
``binding`` marshals arguments to it.  ``catalogs`` holds the seeded synthetic
inputs.  Importing the package does not load the CUDA library; the first call
into ``binding`` does, and fails loudly if it is missing.
"""
