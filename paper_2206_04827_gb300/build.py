"""Build libcyl.so in-tree: nvcc for the CUDA translation units (sm_103a only),
g++ for the host plan, compiled in parallel and linked into
paper_2206_04827_gb300/libcyl.so.  Run as ``python -m paper_2206_04827_gb300.build``."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
OUT_DIR = os.path.join(HERE, '_build')
LIB = os.path.join(HERE, 'libcyl.so')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']


def _nvcc():
    for cand in (os.environ.get('NVCC'), '/usr/local/cuda/bin/nvcc', shutil.which('nvcc')):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError('nvcc not found')


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError('command failed: %s\n%s' % (' '.join(cmd), r.stdout))
    return r.stdout


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(('.cu', '.cpp')))


def build(verbose=False, extra_nvcc=()):
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    inc = ['-I', os.path.join(HERE, '..', 'include'), '-I', CSRC]
    jobs = []
    for src in sources():
        path = os.path.join(CSRC, src)
        obj = os.path.join(OUT_DIR, src + '.o')
        if src.endswith('.cu'):
            cmd = [nvcc, '-O3', '-std=c++17', '-lineinfo', '-Xcompiler', '-fPIC', '-Xptxas', '-v'] + ARCH \
                + list(extra_nvcc) + inc + ['-c', path, '-o', obj]
        else:
            cmd = ['g++', '-O2', '-std=c++17', '-fPIC', '-Wall'] + inc + ['-c', path, '-o', obj]
        jobs.append((cmd, obj))
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        logs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for l in logs:
            sys.stdout.write(l)
    tmp = LIB + '.tmp'
    _run([nvcc, '-shared'] + ARCH + ['-o', tmp] + [o for _, o in jobs] + ['-lcudart_static', '-lrt', '-lpthread', '-ldl'])
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    build(verbose='-v' in sys.argv)
    print(LIB)
