"""GB300 (sm_103a) spatial indexes from "Parallel Dynamic Spatial Indexes"
(PPoPP '26, arXiv 2601.05347): SPaC-Z / SPaC-H and P-Orth trees with batch
build, insert, delete, k-NN, range count and range list, behind the C ABI of
include/psi.h.  ``paper_2601_05347_gb300.psi`` is the Python binding (import it
explicitly; it needs torch); ``gen`` holds the seeded workloads."""
