"""GB300-native sparse LDL^T with pruned-solve variances diag(N^-1) for
INTEGRAL/SPI least-squares normal equations (Bouchet et al., Sec. 3).

The numeric path lives in the CUDA library csrc/ -> libspi_gb300.so, behind
the C ABI of include/spi.h; `spi` is its ctypes binding.
"""
from . import build
from .spi import (Solver, SpiError, spi_measure_peak, spi_analyse, spi_background_fit, spi_inverse_entries, spi_diag_inverse_refined, spi_analyse_multi, spi_default_options, spi_destroy,
                  spi_diag_inverse, spi_diag_inverse_batch, spi_diag_inverse_noalloc, spi_factor, spi_factor_batch, spi_get_etree,
                  spi_get_perm, spi_info, spi_inverse_block, spi_mle_newton, spi_normal_assemble, spi_normal_setup,
                  spi_normal_update, spi_solve, spi_solve_batch, spi_strerror, spi_sync,
                  SPI_PREC_FP64, SPI_PREC_MIXED_FP32, SPI_ORDER_ND, SPI_ORDER_NATURAL, SPI_FIT_LSQ, SPI_FIT_MLE,
                  SPI_PATTERN_MAX)

__all__ = ["build", "Solver", "SpiError", "spi_measure_peak", "spi_analyse", "spi_background_fit", "spi_inverse_entries", "spi_diag_inverse_refined", "spi_analyse_multi", "spi_default_options",
           "spi_destroy", "spi_diag_inverse", "spi_diag_inverse_batch", "spi_diag_inverse_noalloc", "spi_factor", "spi_factor_batch",
           "spi_get_etree", "spi_get_perm", "spi_info", "spi_inverse_block", "spi_mle_newton", "spi_normal_assemble",
           "spi_normal_setup", "spi_normal_update", "spi_solve", "spi_solve_batch",
           "spi_strerror", "spi_sync", "SPI_PREC_FP64", "SPI_PREC_MIXED_FP32", "SPI_ORDER_ND",
           "SPI_ORDER_NATURAL", "SPI_FIT_LSQ", "SPI_FIT_MLE", "SPI_PATTERN_MAX"]
