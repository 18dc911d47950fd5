"""GB300 (sm_103a) split-sweep PPMLR-MHD library: Python binding over the C ABI."""
