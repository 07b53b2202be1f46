"""rAPDB on GB300: the CUDA library and its thin Python binding.

* ``rapdb`` -- ctypes binding of the C ABI in ``include/rapdb.h`` (``Solver``,
  ``BatchedSolver``, ``coupling_pass_noalloc``, ``wait_selftest``); argument
  marshalling only, every step runs in ``librapdb.so``.
* ``build`` -- compiles ``csrc/`` for sm_103a into ``librapdb.so`` (and the
  checked build ``librapdb_checked.so``).
* ``workloads`` -- seeded synthetic problem generators (random QCQPs, the
  paper's construction, kernel-learning forms, batches); data only.
* ``passbench`` -- times the coupling pass alone
  (``python -m paper_2605_29291_gb300.passbench``).
"""
