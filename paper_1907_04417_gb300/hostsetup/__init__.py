"""Host-side input generation: PDE operators, compatible-matching aggregate
maps and smooth vectors.  The output is input data shared by the GPU library
and the oracle; nothing here computes the solve phase."""
from . import aggregation, inputs, problems, smooth  # noqa: F401
