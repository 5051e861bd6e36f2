"""GB300-native NN-corrected DGSEM (arXiv 2207.11571).

The compute path is the CUDA library ``libdgnn.so`` (C ABI declared in
``include/dgnn.h``); ``paper_2207_11571_gb300.dg`` is its thin Python binding.
Importing the package does not load the library; the binding loads it on first
use and raises if it is missing.
"""
