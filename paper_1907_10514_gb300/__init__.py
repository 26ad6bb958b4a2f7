"""GB300-native (sm_103a) trapped-ion timestep: all-pairs Coulomb + linear Paul trap +
Langevin bath + velocity Verlet, behind the C ABI of libiontrap.so (include/iontrap.h).

The Python names are those of the C entry points (see ``native``).  Importing the
package loads libiontrap.so and fails loudly if it has not been built.
"""
from .native import *  # noqa: F401,F403
from .native import IonTrapError, Simulation, make_params  # noqa: F401
