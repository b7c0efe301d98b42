"""GB300 library for the solve phase of the single-hierarchy multiple-vector
aggregation-based AMG (D'Ambra & Vassilevski), used as a CG preconditioner.

* ``amg``       - binding of the C ABI (include/amg.h) to libamg_gb300.so;
* ``autograd``  - torch.autograd.Function whose backward is the adjoint solve;
* ``hostsetup`` - seeded host-side input generation (operators, aggregates,
                  smooth vectors);
* ``build``     - in-tree nvcc build of the CUDA library for sm_103a.
"""
