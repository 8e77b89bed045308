"""Seeded synthetic systems and walkers shared by the CUDA path's tests/bench and the oracle."""
from .system import (System, make_system, make_walkers, config_system, tiny_system,
                     cart_components, excited_determinants, CONFIGS, WALKERS, SCREEN_EPS)
