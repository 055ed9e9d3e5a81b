"""GB300-native two-step high-order compact (2SHOC) Laplacian and explicit RK4
integrator for the nonlinear Schroedinger / Gross-Pitaevskii equation
(arXiv 1109.1027).  The compute path is the CUDA library ``libnlse.so``
(sm_103a) reached through :mod:`paper_1109_1027_gb300.nlse`."""
