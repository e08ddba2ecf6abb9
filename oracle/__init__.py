"""FP64 CPU oracle of the ImEx-ARK pseudospectral phase-field hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
bench's CPU-baseline leg, never by the library. Shares no code with the CUDA
path (see model.py for the readings of the paper it follows).
"""
from .model import Model, elastic_B, h_interp, h_prime, wavenumbers, cubic_stiffness, voigt_to_tensor  # noqa: F401
from .ark import (Tableau, TABLES, euler, ark2_giraldo, ark324l2sa, ark436l2sa, ark_step, advance, chen_shen_euler,  # noqa: F401
                  stability_function, wrms, Controller)
