"""GB300-native sequential-update parallel kinetic Monte Carlo.

Nilmeier & Marian, "A rigorous sequential update strategy for parallel kinetic
Monte Carlo simulation" (arXiv:1403.4674): coloured domains with frozen halos,
a palindromic colour schedule that obeys detailed balance, uniformised
rejection-free domain steps.  The compute path is the sm_103a library
``libkmc_gb300.so`` behind the C ABI of ``include/kmc.h``; ``api`` is its thin
Python binding.
"""
from .api import (KMC_LAUNCH_AUTO, KMC_LAUNCH_CLUSTER, KMC_LAUNCH_GRID, KMC_LAUNCH_THREADS, KMC_OBS_PASS, KMC_OBS_SCHEDULE, KMC_INIT_ALL_UP, KMC_INIT_KEEP, KMC_INIT_PER_REPLICA, KMC_INIT_RANDOM, KMC_RATE_BARKER,  # noqa: F401
                  KMC_RATE_METROPOLIS, KMC_SCHEDULE_FIXED, KMC_SCHEDULE_PALINDROME,
                  KMC_SCHEDULE_RANDOM_PERM, KMC_TIME_EXPECTED, KMC_TIME_EXPONENTIAL, KMC_TIME_HORIZON, Lattice,
                  kmc_create_lattice, kmc_debug_barrier, kmc_destroy, kmc_domain_state,
                  kmc_enable_grad, kmc_get_launch, kmc_get_rate_table, kmc_grad, kmc_grad_nu,
                  kmc_kernel_launches, kmc_domain_side, kmc_lr_estimate, kmc_lr_observable, kmc_observables, kmc_profile, kmc_profile_read, kmc_profile_polls, kmc_reset, kmc_run_schedule, kmc_run_schedule_noalloc,
                  kmc_set_horizon, kmc_set_launch, kmc_set_observation, kmc_set_rate_table, kmc_rate_table_error, kmc_set_replica_params, kmc_set_rates, kmc_sync, kmc_version,
                  Ring, kmc_ring_create, kmc_ring_destroy, kmc_ring_run, kmc_ring_set_rates, kmc_ring_state, ring_passes,
                  KMC_PART_BLOCKS, KMC_PART_STRIPES, Partitioned, kmc_part_create, kmc_part_destroy, kmc_part_run,
                  kmc_part_set_rates, kmc_part_state, part_passes)
from ._lib import KmcError  # noqa: F401
