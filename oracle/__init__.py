"""CPU FP64 oracle of the PFC Newton-Krylov-Schwarz time step.  Test
infrastructure: imported only by tests, the smoke check and the CPU-baseline
leg of bench.py; never by the product library."""
