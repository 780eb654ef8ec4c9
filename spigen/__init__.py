"""Seeded synthetic SPI-like inputs (shared by tests, benchmark and oracle callers)."""
from .synth import (SpiConfig, SpiProblem, BandBatch, TINY, SCALE, BAND, SKY, SKY_FULL, SKY_PIX05, generate,
                    generate_bands, generate_uneven, random_spd, scaled, sky_scaled, uneven_config, N_DET)

__all__ = ["SpiConfig", "SpiProblem", "BandBatch", "TINY", "SCALE", "BAND", "SKY", "SKY_FULL", "SKY_PIX05", "generate",
           "generate_bands", "generate_uneven", "random_spd", "scaled", "sky_scaled", "uneven_config", "N_DET"]
