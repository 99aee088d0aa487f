// hf_runtime.cu - the request loop of include/hf.h: a FIFO of independent
// fracture problems, admitted by free slot and device-memory budget, each
// driven by its own host thread on its own CUDA stream so that the work of
// different requests overlaps on the GPU.  Host code only: every step of a
// request runs through the same calls (and kernels) as a single problem.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/hf.h"

namespace {

template <typename T> std::vector<T> copy_of(const T* p, long long n) {
  return (p && n > 0) ? std::vector<T>(p, p + n) : std::vector<T>();
}

// a request with its own copies of every input array
struct Job {
  int64_t id = 0;
  // mesh
  hf_mesh_desc desc{};
  std::vector<double> xyz, dir_val, neu_traction;
  std::vector<int32_t> elem_nodes, face_elems, neu_face;
  std::vector<int8_t> face_local, face_crackable;
  std::vector<int64_t> dir_dof;
  // problem
  hf_request req{};
  std::vector<int64_t> inj_dofs;
  std::vector<double> inj_weights, U0, P0;
  std::vector<int8_t> alpha0, beta0;
  // outcome
  hf_result res{};
  std::vector<double> U, P;
  std::vector<int8_t> alpha, beta;
  int bypassed = 0;
  bool done = false;
};

}  // namespace

struct hf_runtime {
  hf_runtime_opts opts{};
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::deque<std::shared_ptr<Job>> queue;
  std::unordered_map<int64_t, std::shared_ptr<Job>> jobs;
  std::vector<std::thread> workers;
  int64_t next_id = 1;
  int64_t admitted_bytes = 0, peak_bytes = 0;
  int running = 0, peak_running = 0;
  int64_t completed = 0, failed = 0;
  bool stopping = false;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  // first queued job that fits; the head may be passed only max_bypass times
  std::deque<std::shared_ptr<Job>>::iterator pick() {
    int64_t room = opts.hbm_budget_bytes - admitted_bytes;
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      if ((*it)->res.estimate_bytes <= room) {
        if (it != queue.begin()) queue.front()->bypassed++;
        return it;
      }
      if (it == queue.begin() && (*it)->bypassed >= opts.max_bypass) return queue.end();
    }
    return queue.end();
  }

  void finish(const std::shared_ptr<Job>& j, hf_status s) {
    j->res.status = s;
    j->res.t_done = now();
    j->done = true;
    ++completed;
    if (s != HF_OK) ++failed;
  }

  void run(Job& j, cudaStream_t st) {
    hf_mesh* h = nullptr;
    hf_status s = hf_mesh_create(&j.desc, st, &h);
    const hf_request& r = j.req;
    if (s == HF_OK) s = hf_set_material(h, r.E, r.nu, r.sigma_c, r.delta_c, r.b_stab);
    if (s == HF_OK)
      s = hf_set_injection(h, r.mu, r.Q0, (int64_t)j.inj_dofs.size(), j.inj_dofs.data(),
                           j.inj_weights.empty() ? nullptr : j.inj_weights.data(), r.delta_f, r.dt, r.p_vapor,
                           r.cutoff_on, r.L_ref);
    if (s == HF_OK) s = hf_set_solver(h, &r.solver);
    int64_t nu = 0, np = 0, nfn = 0;
    if (h) hf_get_sizes(h, &nu, &np, &nfn);
    const long long nf = j.desc.n_faces;
    j.res.n_u = nu;
    j.res.n_p = np;
    j.res.n_faces = nf;
    if (s == HF_OK) {
      if (j.U0.empty()) j.U0.assign(nu, 0.0);
      if (j.P0.empty()) j.P0.assign(np, 0.0);
      if (j.alpha0.empty()) j.alpha0.assign(nf, 0);
      if (j.beta0.empty()) j.beta0.assign(nf, 0);
      if ((long long)j.U0.size() != nu || (long long)j.P0.size() != np || (long long)j.alpha0.size() != nf ||
          (long long)j.beta0.size() != nf)
        s = HF_ERR_INVALID_ARG;
      else
        s = hf_set_state(h, j.U0.data(), j.P0.data(), j.alpha0.data(), j.beta0.data(), nullptr, r.t0);
    }
    for (int k = 0; s == HF_OK && k < r.n_steps; ++k) {
      hf_step_report rep{};
      s = hf_advance_step(h, &r.step, &rep);
      j.res.newton_iters += rep.newton_iters;
      j.res.gmres_iters += rep.gmres_iters;
      j.res.cutbacks += rep.cutbacks;
      if (s == HF_OK) j.res.steps_done++;
    }
    if (h) {
      int64_t stt[16] = {0};
      hf_get_stats(h, stt);
      j.res.device_bytes = stt[10];
      j.U.resize(nu);
      j.P.resize(np);
      j.alpha.resize(nf);
      j.beta.resize(nf);
      double t = 0.0;
      hf_status g = hf_get_state(h, j.U.data(), j.P.data(), j.alpha.data(), j.beta.data(), nullptr, &t);
      if (g == HF_OK) j.res.t_final = t;
      if (s == HF_OK) s = g;
      hf_mesh_destroy(h);
    }
    j.res.status = s;
  }

  void worker() {
    cudaSetDevice(opts.device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
      std::shared_ptr<Job> j;
      {
        std::unique_lock<std::mutex> lk(mu);
        work_cv.wait(lk, [&] { return stopping || pick() != queue.end(); });
        if (stopping) break;
        auto it = pick();
        j = *it;
        queue.erase(it);
        admitted_bytes += j->res.estimate_bytes;
        peak_bytes = std::max(peak_bytes, admitted_bytes);
        peak_running = std::max(peak_running, ++running);
        j->res.t_admit = now();
      }
      run(*j, st);
      {
        std::lock_guard<std::mutex> lk(mu);
        admitted_bytes -= j->res.estimate_bytes;
        --running;
        finish(j, j->res.status);
      }
      done_cv.notify_all();
      work_cv.notify_all();
    }
    if (st) cudaStreamDestroy(st);
  }
};

extern "C" {

hf_status hf_runtime_create(const hf_runtime_opts* o, hf_runtime** out) {
  if (!o || !out || o->slots < 1 || o->slots > 64 || o->hbm_budget_bytes <= 0 || o->max_bypass < 0)
    return HF_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o->device < 0 || o->device >= ndev) {
    cudaGetLastError();
    return HF_ERR_CUDA;
  }
  hf_runtime* rt = new hf_runtime();
  rt->opts = *o;
  rt->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < o->slots; ++i) rt->workers.emplace_back([rt] { rt->worker(); });
  *out = rt;
  return HF_OK;
}

hf_status hf_runtime_destroy(hf_runtime* rt) {
  if (!rt) return HF_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(rt->mu);
    rt->stopping = true;
    for (auto& j : rt->queue) rt->finish(j, HF_ERR_STATE);
    rt->queue.clear();
  }
  rt->work_cv.notify_all();
  for (std::thread& t : rt->workers) t.join();
  delete rt;
  return HF_OK;
}

hf_status hf_runtime_submit(hf_runtime* rt, const hf_request* r, int64_t* id) {
  if (!rt || !r || !id || !r->mesh || r->n_steps < 0 || r->n_inj < 0 || (r->n_inj > 0 && !r->inj_dofs))
    return HF_ERR_INVALID_ARG;
  const hf_mesh_desc& d = *r->mesh;
  if ((d.dim != 2 && d.dim != 3) || d.n_nodes <= 0 || d.n_elems <= 0 || d.n_faces <= 0 || !d.xyz || !d.elem_nodes ||
      !d.face_elems || !d.face_local || !d.face_crackable || d.n_dirichlet < 0 || d.n_neumann < 0 ||
      (d.n_dirichlet > 0 && !d.dir_dof) || (d.n_neumann > 0 && (!d.neu_face || !d.neu_traction)))
    return HF_ERR_INVALID_ARG;
  auto j = std::make_shared<Job>();
  const long long dim = d.dim, nen = dim == 2 ? 6 : 10;
  j->xyz = copy_of(d.xyz, d.n_nodes * dim);
  j->elem_nodes = copy_of(d.elem_nodes, d.n_elems * nen);
  j->face_elems = copy_of(d.face_elems, 2 * d.n_faces);
  j->face_local = copy_of(d.face_local, 2 * d.n_faces);
  j->face_crackable = copy_of(d.face_crackable, d.n_faces);
  j->dir_dof = copy_of(d.dir_dof, d.n_dirichlet);
  j->dir_val = copy_of(d.dir_val, d.n_dirichlet);
  j->neu_face = copy_of(d.neu_face, d.n_neumann);
  j->neu_traction = copy_of(d.neu_traction, d.n_neumann * dim);
  j->desc = d;
  j->desc.xyz = j->xyz.data();
  j->desc.elem_nodes = j->elem_nodes.data();
  j->desc.face_elems = j->face_elems.data();
  j->desc.face_local = j->face_local.data();
  j->desc.face_crackable = j->face_crackable.data();
  j->desc.dir_dof = j->dir_dof.empty() ? nullptr : j->dir_dof.data();
  j->desc.dir_val = j->dir_val.empty() ? nullptr : j->dir_val.data();
  j->desc.neu_face = j->neu_face.empty() ? nullptr : j->neu_face.data();
  j->desc.neu_traction = j->neu_traction.empty() ? nullptr : j->neu_traction.data();
  j->req = *r;
  j->req.mesh = &j->desc;
  j->inj_dofs = copy_of(r->inj_dofs, r->n_inj);
  j->inj_weights = copy_of(r->inj_weights, r->n_inj);
  int64_t est = 0, nu = 0, np = 0;
  if (hf_estimate_device_bytes(&j->desc, &r->solver, &est) != HF_OK ||
      hf_mesh_sizes(&j->desc, &nu, &np) != HF_OK)
    return HF_ERR_INVALID_ARG;
  j->alpha0 = copy_of(r->alpha0, d.n_faces);
  j->beta0 = copy_of(r->beta0, d.n_faces);
  j->U0 = copy_of(r->U0, nu);
  j->P0 = copy_of(r->P0, np);
  j->res.estimate_bytes = est;
  std::lock_guard<std::mutex> lk(rt->mu);
  j->id = rt->next_id++;
  j->res.t_submit = rt->now();
  rt->jobs[j->id] = j;
  *id = j->id;
  if (est > rt->opts.hbm_budget_bytes) {
    rt->finish(j, HF_ERR_OOM);
    rt->done_cv.notify_all();
    return HF_OK;
  }
  rt->queue.push_back(j);
  rt->work_cv.notify_one();
  return HF_OK;
}

hf_status hf_runtime_wait(hf_runtime* rt, int64_t id, double timeout_s, hf_result* res) {
  if (!rt) return HF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(rt->mu);
  auto it = rt->jobs.find(id);
  if (it == rt->jobs.end()) return HF_ERR_INVALID_ARG;
  std::shared_ptr<Job> j = it->second;
  if (timeout_s < 0) {
    rt->done_cv.wait(lk, [&] { return j->done; });
  } else if (!rt->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return j->done; })) {
    return HF_ERR_TIMEOUT;
  }
  if (res) *res = j->res;
  return HF_OK;
}

hf_status hf_runtime_fetch(hf_runtime* rt, int64_t id, double* U, double* P, int8_t* alpha, int8_t* beta) {
  if (!rt) return HF_ERR_INVALID_ARG;
  std::shared_ptr<Job> j;
  {
    std::lock_guard<std::mutex> lk(rt->mu);
    auto it = rt->jobs.find(id);
    if (it == rt->jobs.end() || !it->second->done) return HF_ERR_INVALID_ARG;
    j = it->second;
    rt->jobs.erase(it);
  }
  if (U && !j->U.empty()) std::memcpy(U, j->U.data(), j->U.size() * sizeof(double));
  if (P && !j->P.empty()) std::memcpy(P, j->P.data(), j->P.size() * sizeof(double));
  if (alpha && !j->alpha.empty()) std::memcpy(alpha, j->alpha.data(), j->alpha.size());
  if (beta && !j->beta.empty()) std::memcpy(beta, j->beta.data(), j->beta.size());
  return HF_OK;
}

hf_status hf_runtime_stats(hf_runtime* rt, int64_t* st) {
  if (!rt || !st) return HF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(rt->mu);
  int64_t unfetched = 0;
  for (auto& kv : rt->jobs) unfetched += kv.second->done;
  st[0] = (int64_t)rt->queue.size();
  st[1] = rt->running;
  st[2] = unfetched;
  st[3] = rt->admitted_bytes;
  st[4] = rt->peak_bytes;
  st[5] = rt->peak_running;
  st[6] = rt->completed;
  st[7] = rt->failed;
  return HF_OK;
}

double hf_runtime_now(const hf_runtime* rt) { return rt ? rt->now() : 0.0; }

}  // extern "C"
