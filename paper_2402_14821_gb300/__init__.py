"""GB300-native DFF lower-bound feasibility check for the bin_packing constraint
(arXiv 2402.14821).  The CUDA library is loaded lazily by ``binding``."""
