"""CPU FP64 oracle for the stencil programs of the Open Earth Compiler paper.

This package is TEST INFRASTRUCTURE. It is the slow, plain, obviously correct
restatement of what the GPU path computes, written in numpy float64 straight
from the paper's definitions (and, where the paper gives only the shape of a
program, from the readings listed in the project's design notes). It shares no
code with the CUDA path and imports nothing from it. Only the tests, the
package's smoke check and the CPU-baseline leg of the benchmark may import it.

Modules
  stencils  - horizontal diffusion (hdiff), vertical advection (Thomas solve),
              hdiff+vadvc and the fastwaves-like program, staged over the
              inferred bounding boxes (paper §V-B) and per point (inlined,
              paper §V-A).
  program   - parser, shape inference (paper §V-B), staged and inlined
              interpreters for the textual stencil-program form (paper §IV).
  mlp       - FP64 forward/backward/Adam of the cost-model MLP.

Every floating-point expression is evaluated in the order written, in IEEE
binary64 without contraction (numpy never fuses a multiply and an add).
"""

from . import stencils, program, mlp  # noqa: F401
