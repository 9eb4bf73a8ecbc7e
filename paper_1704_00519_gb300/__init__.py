"""GB300 (sm_103a) implementation of the per-stage cut-cell finite-volume
update of the conservative sharp-interface method for compressible
multi-material flows (Pan, Han, Hu & Adams, arXiv:1704.00519).

``paper_1704_00519_gb300.msf`` binds the CUDA library (C ABI in include/msf.h);
``paper_1704_00519_gb300.cases`` builds seeded initial data.
"""
