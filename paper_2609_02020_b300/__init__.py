"""B300-native torque-sampling MPPI (CUDA library for sm_103a + thin binding).

Importing the package loads nothing; ``paper_2609_02020_b300.mppi`` loads the
CUDA library ``libmppi.so`` on first use and raises if it is missing.
"""
