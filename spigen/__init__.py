"""Seeded synthetic SPI-like inputs (shared by tests, benchmark and oracle callers)."""
from .synth import (SpiConfig, SpiProblem, TINY, SCALE, BAND, generate, random_spd,
                    scaled, uneven_config, N_DET)

__all__ = ["SpiConfig", "SpiProblem", "TINY", "SCALE", "BAND", "generate", "random_spd",
           "scaled", "uneven_config", "N_DET"]
